// Ray correction (Sec. 6; Table 7) on the device, complex FP64 throughout.
//
// The near-kernel error is sought as sum_j exp(i k d_j . x) a_j(x) over the eight directions
// d_j = (cos j pi/4, sin j pi/4), with ray functions a_j bilinear on a ray grid of spacing
// H = m h (every m-th node of the fine vertex grid). With P the fine-grid matrix of these basis
// functions (column 8 C + j: the hat of ray node C times plane wave j), the correction is the
// Galerkin projection x += P (P^H A P)^{-1} P^H r of the residual r.
//
// The ray operator couples ray nodes at most one apart, so ordered by rows of ray nodes it is
// block tridiagonal: block row J holds the 8 (nc + 1) unknowns of ray row J (node-major, eight
// directions inner), with blocks L_J (row J - 1), D_J and U_J (row J + 1). It is factored once by
// block LU: S_0 = D_0, S_J = D_J - L_J S_{J-1}^{-1} U_{J-1}, each S_J inverted by Gauss-Jordan
// elimination with row pivoting; the solve keeps S_J^{-1}, G_J = L_J S_{J-1}^{-1} and
// W_J = S_J^{-1} U_J, and runs one step of iterative refinement on the block residual.
//
// Every kernel here is launched with programmatic stream serialization and starts with pdl_enter()
// (hz_common.cuh): it waits for its predecessor before reading anything.
#include "hz_common.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr double RAY_S = 0x1.6a09e667f3bcdp-1;  // sqrt(1/2), correctly rounded

__device__ __forceinline__ void ray_dir(int j, double& dx, double& dy) {
  const double a[8] = {1.0, RAY_S, 0.0, -RAY_S, -1.0, -RAY_S, 0.0, RAY_S};
  const double b[8] = {0.0, RAY_S, 1.0, RAY_S, 0.0, -RAY_S, -1.0, -RAY_S};
  dx = a[j];
  dy = b[j];
}

__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Weight of the bilinear hat of a ray node at fine distance (di, dj); exact for m a power of two.
__device__ __forceinline__ double hat_w(int di, int dj, double rm) {
  return (1.0 - (double)abs(di) * rm) * (1.0 - (double)abs(dj) * rm);
}

// ph[j N + p] = exp(i k (d_x x + d_y y)) at node p = (i, jj), x = i h, y = jj h.
__global__ void ray_phase_kernel(double2* ph, int n, double k) {
  pdl_enter();
  const long long N = (long long)(n + 1) * (n + 1);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 8 * N) return;
  const int j = (int)(t / N);
  const long long p = t - j * N;
  const int i = (int)(p % (n + 1)), jj = (int)(p / (n + 1));
  const double h = 1.0 / n;
  double dx, dy;
  ray_dir(j, dx, dy);
  const double arg = __dmul_rn(k, __dadd_rn(__dmul_rn(dx, __dmul_rn((double)i, h)), __dmul_rn(dy, __dmul_rn((double)jj, h))));
  double s, c;
  sincos(arg, &s, &c);
  ph[t] = make_double2(c, s);
}

// One warp per (column ray node C', direction j', neighbouring ray node C): the eight entries
// (8 C + j, 8 C' + j') of P^H A P, j = 0..7. The sum runs over the fine nodes p under the hat of
// C where A applied to the column (hat of C' times plane wave j') can be non-zero; A's rows are
// the scaled 5-point rows with mirrored boundary neighbours (hz_common.cuh), times 1/h^2.
__global__ void __launch_bounds__(256) ray_assemble_kernel(double2* Lb, double2* Db, double2* Ub, const double2* ph,
                                                           const double* kh, int n, int m) {
  pdl_enter();
  const int nc = n / m, Nr = nc + 1, Bs = 8 * Nr;
  const long long Nc = (long long)Nr * Nr;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= Nc * 72) return;
  const int Cp = (int)(wid / 72), rem = (int)(wid % 72);
  const int jp = rem / 9, q9 = rem % 9;
  const int Ip = Cp % Nr, Jp = Cp / Nr;
  const int I = Ip + q9 % 3 - 1, J = Jp + q9 / 3 - 1;
  if (I < 0 || I > nc || J < 0 || J > nc) return;
  const int i0 = max(max(0, I * m - m + 1), Ip * m - m), i1 = min(min(n, I * m + m - 1), Ip * m + m);
  const int j0 = max(max(0, J * m - m + 1), Jp * m - m), j1 = min(min(n, J * m + m - 1), Jp * m + m);
  const long long N = (long long)(n + 1) * (n + 1);
  const double rm = 1.0 / m;
  const double2* phc = ph + jp * N;
  double ar[8], ai[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) ar[j] = ai[j] = 0.0;
  if (i0 <= i1 && j0 <= j1) {
    const int wi = i1 - i0 + 1, cnt = wi * (j1 - j0 + 1);
    auto col = [&](int a, int c) -> double2 {  // hat of C' times plane wave j' at node (a, c)
      const int di = a - Ip * m, dj = c - Jp * m;
      if (abs(di) >= m || abs(dj) >= m) return make_double2(0.0, 0.0);
      return zscale(phc[(long long)c * (n + 1) + a], hat_w(di, dj, rm));
    };
    for (int q = lane; q < cnt; q += 32) {
      const int i = i0 + q % wi, jj = j0 + q / wi;
      const Nbr b = neighbours(i, jj, n);
      const long long p = (long long)jj * (n + 1) + i;
      const double k1 = kh[p];
      const double2 d = make_double2(k1 * k1 - 4.0, 2.0 * b.sides * k1);
      const double2 s = zadd(zadd(col(b.iw, jj), col(b.ie, jj)), zadd(col(i, b.js), col(i, b.jn)));
      const double2 av = zscale(zadd(s, zmul(d, col(i, jj))), hat_w(i - I * m, jj - J * m, rm));
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const double2 e = zmulc(ph[j * N + p], av);
        ar[j] += e.x;
        ai[j] += e.y;
      }
    }
  }
  const double n2 = (double)n * (double)n;
  double2* blk = Jp == J - 1 ? Lb : (Jp == J ? Db : Ub);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const double re = warp_sum(ar[j]), im = warp_sum(ai[j]);
    if (lane == j) blk[((long long)J * Bs + (8 * I + j)) * Bs + (8 * Ip + jp)] = make_double2(re * n2, im * n2);
  }
}

// g[8 C + j] = sum over the hat of ray node C of hat(p) conj(ph_j[p]) r[p]   (g = P^H r). One warp
// per ray node (eight per block of 256 threads).
__global__ void __launch_bounds__(256) ray_restrict_kernel(double2* g, const double2* r, const double2* ph, int n,
                                                           int m) {
  pdl_enter();
  const int nc = n / m, Nr = nc + 1;
  const long long C = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (C >= (long long)Nr * Nr) return;
  const int I = (int)(C % Nr), J = (int)(C / Nr);
  const int i0 = max(0, I * m - m + 1), i1 = min(n, I * m + m - 1);
  const int j0 = max(0, J * m - m + 1), j1 = min(n, J * m + m - 1);
  const int wi = i1 - i0 + 1, cnt = wi * (j1 - j0 + 1);
  const long long N = (long long)(n + 1) * (n + 1);
  const double rm = 1.0 / m;
  double ar[8], ai[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) ar[j] = ai[j] = 0.0;
  for (int q = lane; q < cnt; q += 32) {
    const int i = i0 + q % wi, jj = j0 + q / wi;
    const long long p = (long long)jj * (n + 1) + i;
    const double2 wr = zscale(r[p], hat_w(i - I * m, jj - J * m, rm));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const double2 e = ph[j * N + p];
      ar[j] = fma(e.x, wr.x, fma(e.y, wr.y, ar[j]));
      ai[j] = fma(e.x, wr.y, fma(-e.y, wr.x, ai[j]));
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const double re = warp_sum(ar[j]), im = warp_sum(ai[j]);
    if (lane == j) g[8 * C + j] = make_double2(re, im);
  }
}

// x[p] += sum_j ph_j[p] * (bilinear interpolation of the ray function z_j at p)   (x += P z)
__global__ void ray_prolong_add_kernel(double2* x, const double2* z, const double2* ph, int n, int m) {
  pdl_enter();
  const long long N = (long long)(n + 1) * (n + 1);
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= N) return;
  const int i = (int)(p % (n + 1)), jj = (int)(p / (n + 1));
  const int Nr = n / m + 1;
  const int I = i / m, ti = i - I * m, J = jj / m, tj = jj - J * m;
  const double rm = 1.0 / m;
  const double wx1 = ti * rm, wx0 = 1.0 - wx1, wy1 = tj * rm, wy0 = 1.0 - wy1;
  const double2* z00 = z + 8LL * ((long long)J * Nr + I);
  double2 tot = make_double2(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    double2 e = zscale(z00[j], wx0 * wy0);
    if (ti) e = zadd(e, zscale(z00[8 + j], wx1 * wy0));
    if (tj) {
      e = zadd(e, zscale(z00[8LL * Nr + j], wx0 * wy1));
      if (ti) e = zadd(e, zscale(z00[8LL * Nr + 8 + j], wx1 * wy1));
    }
    tot = zadd(tot, zmul(ph[j * N + p], e));
  }
  x[p] = zadd(x[p], tot);
}

// Step k of the in-place Gauss-Jordan inversion with row pivoting of the Bs x Bs matrix S: the row
// of largest |S[i][k]| (i >= k; the first on ties) is swapped into row k and recorded in perm[k];
// column k is saved in fcol; row k is scaled by 1 / pivot with the pivot's own entry replaced by
// 1 / pivot. A zero or non-finite pivot column sets *status = 1 (the inverse is then meaningless).
__global__ void __launch_bounds__(1024) ray_gj_pivot_kernel(double2* S, int Bs, int k, double2* fcol, int* perm,
                                                            int* status) {
  pdl_enter();
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ int piv;
  double best = -1.0;
  int bi = Bs;
  for (int i = k + threadIdx.x; i < Bs; i += blockDim.x) {
    const double2 a = S[(long long)i * Bs + k];
    const double v = a.x * a.x + a.y * a.y;
    if (v > best) {
      best = v;
      bi = i;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[warp] = best;
    si[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = -1.0;
    int ib = Bs;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (sv[w] > b || (sv[w] == b && si[w] < ib)) {
        b = sv[w];
        ib = si[w];
      }
    }
    const bool ok = b > 0.0 && isfinite(b) && ib < Bs;
    if (!ok) *status = 1;
    piv = ok ? ib : k;
    perm[k] = piv;
  }
  __syncthreads();
  const int p = piv;
  if (p != k) {
    for (int c = threadIdx.x; c < Bs; c += blockDim.x) {
      const double2 t = S[(long long)k * Bs + c];
      S[(long long)k * Bs + c] = S[(long long)p * Bs + c];
      S[(long long)p * Bs + c] = t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Bs; i += blockDim.x) fcol[i] = S[(long long)i * Bs + k];
  __syncthreads();
  const double2 pv = fcol[k];
  const double d = pv.x * pv.x + pv.y * pv.y;
  const double2 inv = make_double2(pv.x / d, -pv.y / d);
  for (int c = threadIdx.x; c < Bs; c += blockDim.x) {
    const long long q = (long long)k * Bs + c;
    S[q] = c == k ? inv : zmul(S[q], inv);
  }
}

// Rows i != k: S[i][c] = (c == k ? 0 : S[i][c]) - fcol[i] S[k][c]  (row k is only read).
__global__ void ray_gj_elim_kernel(double2* S, int Bs, int k, const double2* fcol) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (c >= Bs || i == k) return;
  const double2 f = fcol[i];
  if (f.x == 0.0 && f.y == 0.0) return;  // the row already holds its final values (S[i][k] is 0)
  const long long q = (long long)i * Bs + c;
  const double2 a = c == k ? make_double2(0.0, 0.0) : S[q];
  const double2 fr = zmul(f, S[(long long)k * Bs + c]);
  S[q] = make_double2(a.x - fr.x, a.y - fr.y);
}

// Undo the row interchanges on the inverse: columns k and perm[k] swapped, k = Bs-1 .. 0.
__global__ void ray_gj_unpermute_kernel(double2* S, int Bs, const int* perm) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bs) return;
  double2* row = S + (long long)i * Bs;
  for (int k = Bs - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      const double2 t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
}

// C = A B (acc 0) or C = C - A B (acc 1) for Bs x Bs row-major blocks; C aliases neither A nor B.
// A 32 x 32 tile of C per block of 256 threads, each thread 2 x 2 entries, k in steps of 16.
__global__ void __launch_bounds__(256) ray_gemm_kernel(double2* C, const double2* A, const double2* B, int Bs,
                                                       int acc) {
  pdl_enter();
  __shared__ double2 As[32][17];
  __shared__ double2 Bsh[16][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
  double2 c[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) c[a][b] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < Bs; k0 += 16) {
    for (int e = threadIdx.x; e < 512; e += 256) {
      const int r = e >> 4, kk = e & 15, gr = row0 + r, gk = k0 + kk;
      As[r][kk] = (gr < Bs && gk < Bs) ? A[(long long)gr * Bs + gk] : make_double2(0.0, 0.0);
      const int kb = e >> 5, cc = e & 31, gk2 = k0 + kb, gc = col0 + cc;
      Bsh[kb][cc] = (gk2 < Bs && gc < Bs) ? B[(long long)gk2 * Bs + gc] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      const double2 a0 = As[ty][kk], a1 = As[ty + 16][kk], b0 = Bsh[kk][tx], b1 = Bsh[kk][tx + 16];
      c[0][0] = zadd(c[0][0], zmul(a0, b0));
      c[0][1] = zadd(c[0][1], zmul(a0, b1));
      c[1][0] = zadd(c[1][0], zmul(a1, b0));
      c[1][1] = zadd(c[1][1], zmul(a1, b1));
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int r = row0 + ty + 16 * a, cc = col0 + tx + 16 * b;
      if (r < Bs && cc < Bs) {
        const long long q = (long long)r * Bs + cc;
        C[q] = acc ? make_double2(C[q].x - c[a][b].x, C[q].y - c[a][b].y) : c[a][b];
      }
    }
}

// out_b = base_b + sgn M_b x_b for b = blockIdx.y (M_b advances Bs^2 entries, the vectors Bs);
// base may be null (zero) or equal to out; x aliases neither. One block of GEMV_THREADS per row
// (blockIdx.x): GB300's FP64 pipe is narrow, so a row is spread over four warps to keep every SM
// sub-partition busy, and each complex product is accumulated with four FMAs.
constexpr int GEMV_THREADS = 128;
__global__ void __launch_bounds__(GEMV_THREADS) ray_gemv_kernel(double2* out, const double2* base, const double2* M,
                                                                const double2* x, int Bs, double sgn) {
  pdl_enter();
  const int row = blockIdx.x;
  const long long b = blockIdx.y;
  const double2* Mr = M + b * Bs * (long long)Bs + (long long)row * Bs;
  const double2* xb = x + b * Bs;
  double re = 0.0, im = 0.0;
  for (int c0 = threadIdx.x; c0 < Bs; c0 += 4 * GEMV_THREADS) {
    double2 a[4], v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + GEMV_THREADS * u;
      a[u] = c < Bs ? Mr[c] : make_double2(0.0, 0.0);
      v[u] = c < Bs ? xb[c] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      re = fma(a[u].x, v[u].x, re);
      re = fma(-a[u].y, v[u].y, re);
      im = fma(a[u].x, v[u].y, im);
      im = fma(a[u].y, v[u].x, im);
    }
  }
  re = warp_sum(re);
  im = warp_sum(im);
  __shared__ double red[2][GEMV_THREADS / 32];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = re;
    red[1][warp] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int w = 0; w < GEMV_THREADS / 32; ++w) {
      sr += red[0][w];
      si += red[1][w];
    }
    const double2 o = base ? base[b * Bs + row] : make_double2(0.0, 0.0);
    out[b * Bs + row] = make_double2(o.x + sgn * sr, o.y + sgn * si);
  }
}

// e_J = g_J - (L_J z_{J-1} + D_J z_J + U_J z_{J+1}), one thread per row of the whole system. Row
// 8 I + j of block row J couples only ray nodes I - 1 .. I + 1 of the three ray rows, so only those
// 24 columns of each block are read (the others are zero by construction).
__global__ void __launch_bounds__(128) ray_block_residual_kernel(double2* e, const double2* g, const double2* z,
                                                                 const double2* Lb, const double2* Db,
                                                                 const double2* Ub, int Bs, int Nr) {
  pdl_enter();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)Nr * Bs) return;
  const int J = (int)(t / Bs), row = (int)(t % Bs), I = row / 8;
  const int c0 = 8 * max(I - 1, 0), c1 = 8 * min(I + 2, Nr);
  const long long off = (long long)J * Bs * Bs + (long long)row * Bs;
  const double2* zJ = z + (long long)J * Bs;
  double re = 0.0, im = 0.0;
  for (int c = c0; c < c1; ++c) {
    double2 q = zmul(Db[off + c], zJ[c]);
    if (J > 0) q = zadd(q, zmul(Lb[off + c], zJ[c - Bs]));
    if (J < Nr - 1) q = zadd(q, zmul(Ub[off + c], zJ[c + Bs]));
    re += q.x;
    im += q.y;
  }
  e[t] = make_double2(g[t].x - re, g[t].y - im);
}

__global__ void ray_copy_kernel(double2* dst, const double2* src, int cnt) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) dst[i] = src[i];
}

constexpr int RED_BLOCKS = 512, RED_THREADS = 256;

// r = b - v and per-block partial sums of |r|^2 (v null: |b|^2 only, r untouched).
__global__ void __launch_bounds__(RED_THREADS) ray_residual_norm_kernel(double2* r, const double2* b, const double2* v,
                                                                        long long N, double* partials) {
  pdl_enter();
  double s = 0.0;
  for (long long p = blockIdx.x * (long long)RED_THREADS + threadIdx.x; p < N; p += (long long)RED_BLOCKS * RED_THREADS) {
    double2 t = b[p];
    if (v) {
      const double2 w = v[p];
      t = make_double2(t.x - w.x, t.y - w.y);
      r[p] = t;
    }
    s += t.x * t.x + t.y * t.y;
  }
  __shared__ double red[RED_THREADS / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void ray_sum_kernel(const double* partials, double* out) {
  pdl_enter();
  __shared__ double red[RED_BLOCKS];
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) red[i] = partials[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < RED_BLOCKS; ++i) t += red[i];
    *out = t;
  }
}

__global__ void ray_axpy_kernel(double2* x, const double2* z, long long N) {
  pdl_enter();
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p < N) x[p] = zadd(x[p], z[p]);
}

inline unsigned blocks_for(long long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------- launchers

cudaError_t launch_ray_phases(double2* ph, int n, double k, cudaStream_t s) {
  const long long work = 8LL * (n + 1) * (n + 1);
  return pdl_launch(ray_phase_kernel, dim3(blocks_for(work, 256)), dim3(256), 0, s, ph, n, k);
}

cudaError_t launch_ray_assemble(const RayBlocks& B, const double2* ph, const double* kh, cudaStream_t s) {
  const long long warps = 72LL * B.Nr * B.Nr;
  return pdl_launch(ray_assemble_kernel, dim3(blocks_for(warps * 32, 256)), dim3(256), 0, s, B.L, B.D, B.U, ph, kh,
                    B.n, B.m);
}

cudaError_t launch_ray_restrict(double2* g, const double2* r, const double2* ph, int n, int m, cudaStream_t s) {
  const long long Nr = n / m + 1;
  return pdl_launch(ray_restrict_kernel, dim3(blocks_for(32 * Nr * Nr, 256)), dim3(256), 0, s, g, r, ph, n, m);
}

cudaError_t launch_ray_prolong_add(double2* x, const double2* z, const double2* ph, int n, int m, cudaStream_t s) {
  return pdl_launch(ray_prolong_add_kernel, dim3(blocks_for((long long)(n + 1) * (n + 1), 256)), dim3(256), 0, s, x,
                    z, ph, n, m);
}

namespace {

cudaError_t gj_inverse(double2* S, int Bs, double2* fcol, int* perm, int* status, cudaStream_t s) {
  const dim3 eg(blocks_for(Bs, 128), Bs);
  for (int k = 0; k < Bs; ++k) {
    cudaError_t e = pdl_launch(ray_gj_pivot_kernel, dim3(1), dim3(1024), 0, s, S, Bs, k, fcol, perm, status);
    if (e == cudaSuccess) e = pdl_launch(ray_gj_elim_kernel, eg, dim3(128), 0, s, S, Bs, k, (const double2*)fcol);
    if (e != cudaSuccess) return e;
  }
  return pdl_launch(ray_gj_unpermute_kernel, dim3(blocks_for(Bs, 128)), dim3(128), 0, s, S, Bs, (const int*)perm);
}

cudaError_t gemm(double2* C, const double2* A, const double2* Bm, int Bs, int acc, cudaStream_t s) {
  const dim3 g(blocks_for(Bs, 32), blocks_for(Bs, 32));
  return pdl_launch(ray_gemm_kernel, g, dim3(256), 0, s, C, A, Bm, Bs, acc);
}

cudaError_t gemv(double2* out, const double2* base, const double2* M, const double2* x, int Bs, int batch, double sgn,
                 cudaStream_t s) {
  return pdl_launch(ray_gemv_kernel, dim3(Bs, batch), dim3(GEMV_THREADS), 0, s, out, base, M, x, Bs, sgn);
}

// z = (block LU)^{-1} g; y is scratch of one vector.
cudaError_t block_substitute(const RayBlocks& B, double2* z, const double2* g, double2* y, cudaStream_t s) {
  const int Bs = B.Bs, Nr = B.Nr;
  const long long bs2 = (long long)Bs * Bs;
  cudaError_t e = pdl_launch(ray_copy_kernel, dim3(blocks_for(Bs, 128)), dim3(128), 0, s, y, g, Bs);
  for (int J = 1; J < Nr && e == cudaSuccess; ++J)
    e = gemv(y + (long long)J * Bs, g + (long long)J * Bs, B.G + J * bs2, y + (long long)(J - 1) * Bs, Bs, 1, -1.0, s);
  if (e == cudaSuccess) e = gemv(z, nullptr, B.Sinv, y, Bs, Nr, 1.0, s);
  for (int J = Nr - 2; J >= 0 && e == cudaSuccess; --J)
    e = gemv(z + (long long)J * Bs, z + (long long)J * Bs, B.W + J * bs2, z + (long long)(J + 1) * Bs, Bs, 1, -1.0, s);
  return e;
}

}  // namespace

cudaError_t ray_factor(const RayBlocks& B, cudaStream_t s) {
  const int Bs = B.Bs, Nr = B.Nr;
  const long long bs2 = (long long)Bs * Bs;
  cudaError_t e = cudaMemcpyAsync(B.Sinv, B.D, sizeof(double2) * (size_t)(bs2 * Nr), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  e = gj_inverse(B.Sinv, Bs, B.fcol, B.perm, B.status, s);
  if (e != cudaSuccess) return e;
  for (int J = 1; J < Nr; ++J) {
    double2* Sprev = B.Sinv + (J - 1) * bs2;
    double2* Sj = B.Sinv + J * bs2;
    if ((e = gemm(B.W + (J - 1) * bs2, Sprev, B.U + (J - 1) * bs2, Bs, 0, s)) != cudaSuccess) return e;
    if ((e = gemm(Sj, B.L + J * bs2, B.W + (J - 1) * bs2, Bs, 1, s)) != cudaSuccess) return e;
    if ((e = gemm(B.G + J * bs2, B.L + J * bs2, Sprev, Bs, 0, s)) != cudaSuccess) return e;
    if ((e = gj_inverse(Sj, Bs, B.fcol, B.perm, B.status, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t ray_coarse_solve(const RayBlocks& B, double2* z, const double2* g, cudaStream_t s) {
  cudaError_t e = block_substitute(B, z, g, B.y, s);
  if (e != cudaSuccess) return e;
  // one step of iterative refinement: z += (block LU)^{-1} (g - A_ray z)
  const long long cnt = (long long)B.Bs * B.Nr;
  e = pdl_launch(ray_block_residual_kernel, dim3(blocks_for(cnt, 128)), dim3(128), 0, s, B.e, g, (const double2*)z,
                 (const double2*)B.L, (const double2*)B.D, (const double2*)B.U, B.Bs, B.Nr);
  if (e == cudaSuccess) e = block_substitute(B, B.dz, B.e, B.y, s);
  if (e == cudaSuccess) e = pdl_launch(ray_axpy_kernel, dim3(blocks_for(cnt, 256)), dim3(256), 0, s, z, (const double2*)B.dz, cnt);
  return e;
}

cudaError_t launch_ray_residual_norm(double2* r, const double2* b, const double2* v, long long N, double* partials,
                                     double* out, cudaStream_t s) {
  cudaError_t e = pdl_launch(ray_residual_norm_kernel, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, r, b, v, N, partials);
  if (e == cudaSuccess) e = pdl_launch(ray_sum_kernel, dim3(1), dim3(256), 0, s, (const double*)partials, out);
  return e;
}

cudaError_t launch_ray_axpy(double2* x, const double2* z, long long N, cudaStream_t s) {
  return pdl_launch(ray_axpy_kernel, dim3(blocks_for(N, 256)), dim3(256), 0, s, x, z, N);
}

int ray_reduction_blocks() { return RED_BLOCKS; }

}  // namespace hz
