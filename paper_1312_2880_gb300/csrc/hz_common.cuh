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

// Programmatic dependent launch: every kernel is launched allowed to start while its predecessor
// in the stream (or graph) is still running. It first waits until the predecessor has completed
// and its writes are visible (griddepcontrol.wait; nothing is read before), then allows its own
// successor to begin launching, so launch latency overlaps execution. Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

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

// Conversions between binary64 and binary32 on the integer pipe. GB300 runs hardware float
// conversions on its narrow FP64 pipe, which the FP32 V-cycle would otherwise saturate just
// reading and writing the FP64 Krylov vectors. Written from the IEEE 754 formats: narrowing
// rounds to nearest, ties to even, on the 29 dropped significand bits (a carry into the exponent
// is the correct rounding); results below the binary32 normal range become signed zero;
// overflow gives infinity; NaN stays NaN. Widening is exact for normal numbers and zero
// (subnormal binary32 inputs become signed zero).
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0x7FF) return __int_as_float((int)(sign | 0x7F800000u | ((b & 0x000FFFFFFFFFFFFFull) ? 0x400000u : 0u)));
  const int ef = e - 1023 + 127;
  if (ef <= 0) return __int_as_float((int)sign);
  const unsigned int m = (unsigned int)((b >> 29) & 0x7FFFFFu);
  const unsigned int rem = (unsigned int)(b & 0x1FFFFFFFu);
  unsigned int mag = ((unsigned int)ef << 23) | m;
  mag += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  if (mag >= 0x7F800000u) mag = 0x7F800000u;
  return __int_as_float((int)(sign | mag));
}
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = (unsigned int)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned int e = (u >> 23) & 0xFF;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long eb = (e == 0xFF) ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (eb << 52) | m));
}

// Load a complex element stored as double2 or float2 and convert it to precision T.
template <class T>
__device__ __forceinline__ c2<T> ldc(const double2* p, long long i) {
  double2 v = p[i];
  return mk<T>((T)v.x, (T)v.y);
}
template <>
__device__ __forceinline__ c2<float> ldc<float>(const double2* p, long long i) {
  double2 v = p[i];
  return mk<float>(f64_to_f32(v.x), f64_to_f32(v.y));
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
template <>
__device__ __forceinline__ void stc<float>(double2* p, long long i, c2<float> v) {
  p[i] = make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
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
// 1/x: IEEE division in FP64; the correctly rounded single-precision reciprocal in FP32.
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }

template <class T>
__device__ __forceinline__ c2<T> cdiv(c2<T> a, c2<T> b) {
  T inv = rcp(b.x * b.x + b.y * b.y);
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

// Fixed-rounding complex arithmetic for the fused Gauss-Seidel passes. Every operation is an
// explicit round-to-nearest add, multiply or fused multiply-add, so the compiler cannot contract
// or reorder it differently from one kernel to another: the tile and streaming forms of a pass,
// which share these helpers and take the same operations in the same order on every node, give
// bit-identical results, and the choice between them never changes a solution.
namespace xr {
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
// FP32: the hardware reciprocal approximation (rcp.approx, about 1 ulp); the divisors here are
// |d|^2 of a Helmholtz diagonal, never denormal. FP64: the correctly rounded reciprocal.
__device__ __forceinline__ float rcp(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }

template <class T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) { return mk<T>(add(a.x, b.x), add(a.y, b.y)); }
template <class T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) { return mk<T>(sub(a.x, b.x), sub(a.y, b.y)); }
template <class T> __device__ __forceinline__ c2<T> cscale(c2<T> a, T s) { return mk<T>(mul(a.x, s), mul(a.y, s)); }
template <class T>
__device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, -mul(a.y, b.y)), fma(a.x, b.y, mul(a.y, b.x)));
}
// conj(a) * b
template <class T>
__device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {
  return mk<T>(fma(a.x, b.x, mul(a.y, b.y)), fma(a.x, b.y, -mul(a.y, b.x)));
}
template <class T> __device__ __forceinline__ T cabs2(c2<T> a) { return fma(a.x, a.x, mul(a.y, a.y)); }
template <class T>
__device__ __forceinline__ c2<T> cdiv(c2<T> a, c2<T> d) {
  const T inv = rcp(fma(d.x, d.x, mul(d.y, d.y)));
  return mk<T>(mul(fma(a.x, d.x, mul(a.y, d.y)), inv), mul(fma(a.y, d.x, -mul(a.x, d.y)), inv));
}
// Scaled-row diagonal (k H)^2 - 4 + i (beta (k H)^2 + 2 sides k H); two_sides = 2 sides.
template <class T>
__device__ __forceinline__ c2<T> diag2(T kh, T two_sides, T beta) {
  const T k2 = mul(kh, kh);
  return mk<T>(sub(k2, (T)4), fma(two_sides, kh, mul(beta, k2)));
}
template <class T>
__device__ __forceinline__ c2<T> diag(T kh, int sides, T beta) { return diag2<T>(kh, (T)(2 * sides), beta); }
// Sum of a node's four neighbours in the order (W + E) + (S + N).
template <class T>
__device__ __forceinline__ c2<T> nb4(c2<T> w, c2<T> e, c2<T> s, c2<T> n) {
  return cadd<T>(cadd<T>(w, e), cadd<T>(s, n));
}
// Gauss-Seidel point update (f - nb) / d and residual f - (d u + nb).
template <class T>
__device__ __forceinline__ c2<T> gs(c2<T> f, c2<T> nb, c2<T> d) { return cdiv<T>(csub<T>(f, nb), d); }
template <class T>
__device__ __forceinline__ c2<T> resid(c2<T> f, c2<T> u, c2<T> nb, c2<T> d) {
  return csub<T>(f, cadd<T>(cmul<T>(d, u), nb));
}
// One row of full weighting: (w + e) + 2 c.
template <class T>
__device__ __forceinline__ c2<T> fw3(c2<T> w, c2<T> c, c2<T> e) { return cadd<T>(cadd<T>(w, e), cscale<T>(c, (T)2)); }
// Full weighting at coarse node (I, J) of a fine array r (row pitch pr, n intervals), fine nodes
// outside the square mirrored: rows (w + e) + 2 c, then across rows the same, times 4/16 (the
// restricted residual is scaled by (2h)^2 / h^2 = 4 for the coarse level's h^2-scaled rows).
template <class T>
__device__ __forceinline__ c2<T> fw_node(const c2<T>* r, int pr, int n, int I, int J) {
  c2<T> row[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const c2<T>* rr = r + (long long)reflect(2 * J + b - 1, n) * pr;
    row[b] = fw3<T>(rr[reflect(2 * I - 1, n)], rr[2 * I], rr[reflect(2 * I + 1, n)]);
  }
  return cscale<T>(fw3<T>(row[0], row[1], row[2]), (T)0.25);
}
// Bilinear interpolation of the coarse correction at fine node (2I + oi, 2J + oj) from coarse rows
// e0 (J) and e1 (J + 1): coincident nodes copy, edge midpoints average two, centres four, in the
// order ((e00 + e10) + (e01 + e11)) / 4.
template <class T>
__device__ __forceinline__ c2<T> bilinear(const c2<T>* e0, const c2<T>* e1, int I, int oi, int oj) {
  if (oi && oj) return cscale<T>(cadd<T>(cadd<T>(e0[I], e1[I]), cadd<T>(e0[I + 1], e1[I + 1])), (T)0.25);
  if (oi) return cscale<T>(cadd<T>(e0[I], e0[I + 1]), (T)0.5);
  if (oj) return cscale<T>(cadd<T>(e0[I], e1[I]), (T)0.5);
  return e0[I];
}
}  // namespace xr

}  // namespace hz
