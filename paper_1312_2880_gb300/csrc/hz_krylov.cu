// Bi-CGSTAB (van der Vorst 1992) in complex FP64 with the preconditioner applied on the right,
// as the outer iteration of Sec. 6: every vector update is fused with the dot products it
// feeds, and the scalars (alpha, omega, beta, rho) are computed on the device by the last
// block of each reduction, so an iteration needs no host round trip and can be replayed from
// a CUDA graph.
//
// The iteration runs on the h^2-scaled system (h^2 L^h) x = h^2 b; x is unchanged and relative
// residuals are scale-free. Reductions are deterministic: each thread sums a fixed set of
// elements in a fixed order, warps and blocks combine in a fixed tree, and the last block adds
// the per-block partials in block order.
#include <cuda_runtime.h>
#include <math.h>

#include "hz_common.cuh"
#include "hz_internal.h"

namespace hz {

namespace {

constexpr int KB = 256;  // threads per block of every Krylov kernel

__device__ __forceinline__ double2 d2add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// a + s * b (complex s)
__device__ __forceinline__ double2 d2axpy(double2 a, double2 s, double2 b) {
  return make_double2(fma(s.x, b.x, fma(-s.y, b.y, a.x)), fma(s.x, b.y, fma(s.y, b.x, a.y)));
}
// a - s * b (complex s)
__device__ __forceinline__ double2 d2axmy(double2 a, double2 s, double2 b) {
  return make_double2(fma(-s.x, b.x, fma(s.y, b.y, a.x)), fma(-s.x, b.y, fma(-s.y, b.x, a.y)));
}
__device__ __forceinline__ double2 d2div(double2 a, double2 b) {
  double inv = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
__device__ __forceinline__ double2 d2mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// Preconditioned vectors: FP64, or FP32 widened exactly (integer pipe, see f32_to_f64).
__device__ __forceinline__ double2 ldy(const double2* p, int e) { return p[e]; }
__device__ __forceinline__ double2 ldy(const float2* p, int e) {
  float2 v = p[e];
  return make_double2(f32_to_f64(v.x), f32_to_f64(v.y));
}
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(f32_to_f64(v.x), f32_to_f64(v.y)); }
// FP64 value rounded to FP32 for the FP32 V-cycle (integer pipe, see f64_to_f32).
__device__ __forceinline__ float2 narrow(double2 v) { return make_float2(f64_to_f32(v.x), f64_to_f32(v.y)); }

__device__ __forceinline__ bool fin(double v) { return isfinite(v); }
__device__ __forceinline__ bool fin2(double2 v) { return isfinite(v.x) && isfinite(v.y); }

template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Sum over the block in a fixed order; the result is valid in thread 0. Every thread stores its
// values, lane L of warp 0 adds column L over the KB / 32 warps, then a shuffle tree. GB300's
// FP64 pipe executes every lane of a warp instruction, so a shuffle tree in each of the KB / 32
// warps costs as much FP64 issue as the kernel's own arithmetic on small grids (measured: the
// reduction of an update at n = 512 took 8.6 us of 31); summing through shared memory first
// leaves one warp's adds per block.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sm)[KB]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) sm[k][threadIdx.x] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = sm[k][lane];
#pragma unroll
      for (int w = 1; w < KB / 32; ++w) s += sm[k][w * 32 + lane];
      v[k] = s;
    }
    warp_sum<NV>(v);
  }
}

// Grid-wide sum. Every block stores its partial; the block that arrives last adds all partials
// in block order and returns true with the totals in `tot` (in every thread of that block).
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* ticket, double (&tot)[NV]) {
  __shared__ double sm[NV][KB];
  __shared__ int is_last;
  __shared__ double res[NV];
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    w[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += KB) w[k] += __ldcg(&partials[k * gridDim.x + b]);
  }
  block_sum<NV>(w, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) res[k] = w[k];
    *ticket = 0;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = res[k];
  return true;
}

// (h^2 A y) at node (i, j) = flat index e of the finest grid (pitch n+1), A = L (beta = 0) or M.
// The FP64 pipe bounds these kernels, so interior nodes of L take the real-diagonal path:
// d = (kh)^2 - 4 (one FMA) and v = nb + d y (two FMAs); boundary nodes and M use the complex row.
// Boundary rows and the shifted operator M: the complex diagonal. Out of line, so that the
// compiler never evaluates this branch's FP64 arithmetic for interior nodes (it is taken by 4n of
// (n+1)^2 nodes; with the branch if-converted the apply kernels were measured 1.65x slower).
template <class Y2>
__device__ __noinline__ double2 apply_row(const Y2* __restrict__ y, double k, int e, int sides, double beta,
                                          double2 nb) {
  double2 d = row_diag<double>(k, sides, beta);
  return d2add(d2mul(d, ldy(y, e)), nb);
}

template <class Y2>
__device__ __forceinline__ double2 apply_at(const Y2* __restrict__ y, const double* __restrict__ kh, int e, int i,
                                            int j, int n, double beta) {
  const int w = n + 1;
  Nbr b = neighbours(i, j, n);
  double2 nb = d2add(d2add(ldy(y, j * w + b.iw), ldy(y, j * w + b.ie)), d2add(ldy(y, b.js * w + i), ldy(y, b.jn * w + i)));
  const double k = kh[e];
  if (b.sides == 0 && beta == 0.0) {
    const double2 ye = ldy(y, e);
    const double dr = fma(k, k, -4.0);
    return make_double2(fma(dr, ye.x, nb.x), fma(dr, ye.y, nb.y));
  }
  return apply_row(y, k, e, b.sides, beta, nb);
}

// Grid-stride walk over the (n+1)^2 nodes that keeps (i, j) up to date without dividing per node.
struct NodeWalk {
  int e, i, j, di, dj, w, stride;
  __device__ __forceinline__ NodeWalk(int n, int stride_) : w(n + 1), stride(stride_) {
    e = blockIdx.x * blockDim.x + threadIdx.x;
    j = e / w;
    i = e - j * w;
    dj = stride / w;
    di = stride - dj * w;
  }
  __device__ __forceinline__ void next() {
    e += stride;
    i += di;
    j += dj;
    if (i >= w) {
      i -= w;
      ++j;
    }
  }
};

__device__ __forceinline__ void hist_push(KState* st, double* hist, double v) {
  if (st->hist_len < st->hist_cap) hist[st->hist_len] = v;
  st->hist_len += 1;
}

#define GRID_STRIDE(e, N) for (int e = blockIdx.x * KB + threadIdx.x; e < (N); e += gridDim.x * KB)

__host__ __device__ __forceinline__ KrylovVecs offset_instance(KrylovVecs k, long long b) {
  if (b) {
    const long long o = b * k.sv;
    k.x += o; k.r += o; k.p += o; k.v += o; k.s += o; k.t += o; k.y += o; k.z += o; k.tr += o; k.b += o;
    k.rhat += o;
    if (k.p32) { k.p32 += o; k.s32 += o; k.y32 += o; k.z32 += o; }
    k.st += b;
    k.partials += b * k.part_stride;
    k.hist += b * k.hist_stride;
  }
  return k;
}
// This block's instance (blockIdx.z).
__device__ __forceinline__ KrylovVecs instance(const KrylovVecs& k) { return offset_instance(k, blockIdx.z); }

// Counter-based SplitMix64 (Steele, Lea, Flood 2014): output number c + 1 of the generator started
// from `seed`, top 53 bits mapped to [0, 1); r^_p = (u_2p - 1/2) + i (u_2p+1 - 1/2).
__device__ __forceinline__ double2 shadow_value(unsigned long long seed, long long p) {
  double u[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(2 * p + c + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    u[c] = (double)(z >> 11) * 0x1.0p-53;
  }
  return make_double2(u[0] - 0.5, u[1] - 0.5);
}

// x = 0, r = h^2 b, p = v = 0, r^ = the first shadow residual (a restart in an earlier solve may
// have renewed it, and every solve starts from the same one); |r|^2 and <r^, r> start the iteration.
__global__ void k_init_kernel(KrylovVecs k, double tol, int maxit, int hist_cap) {
  pdl_enter();
  k = instance(k);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int N = (int)k.N;
  GRID_STRIDE(e, N) {
    double2 bv = k.b[e];
    double2 r = make_double2(bv.x * k.scale_b, bv.y * k.scale_b);
    const double2 rh = shadow_value(SHADOW_SEED, e);
    k.rhat[e] = rh;
    k.r[e] = r;
    k.x[e] = make_double2(0, 0);
    k.p[e] = make_double2(0, 0);
    k.v[e] = make_double2(0, 0);
    acc[0] = fma(r.x, r.x, fma(r.y, r.y, acc[0]));
    acc[1] = fma(rh.x, r.x, fma(rh.y, r.y, acc[1]));
    acc[2] = fma(rh.x, r.y, fma(-rh.y, r.x, acc[2]));
    acc[3] = fma(rh.x, rh.x, fma(rh.y, rh.y, acc[3]));
  }
  double tot[4];
  if (!grid_sum<4>(acc, k.partials, &k.st->ticket[KT_INIT], tot)) return;
  if (threadIdx.x == 0) {
    KState* st = k.st;
    st->bnorm2 = tot[0];
    st->tol2 = tol * tol * tot[0];
    st->rr = tot[0];
    st->rho = make_double2(tot[1], tot[2]);
    st->rho_old = make_double2(1, 0);
    st->alpha = make_double2(1, 0);
    st->omega = make_double2(1, 0);
    st->beta = make_double2(0, 0);
    st->alpha_x = make_double2(0, 0);
    st->omega_x = make_double2(0, 0);
    st->xa = 0;
    st->xw = 0;
    st->first = 1;
    st->half = 0;
    st->it = 1;
    st->hist_len = 0;
    st->hist_cap = hist_cap;
    st->maxit = maxit;
    st->done = 0;
    st->iters_x2 = 0;
    st->shadow_restarts = 0;
    st->rhat2 = tot[3];
    st->min_cos2 = 1.0;
    st->min_step2 = 1.0;
    st->stall_cos2 = k.stall_cos2;
    st->stall_step2 = k.stall_step2;
    st->max_shadow_restarts = k.max_shadow_restarts;
    if (!fin(tot[0]) || !fin(tot[1]) || !fin(tot[2])) st->done = 3;
    else if (tot[0] == 0.0) st->done = 1;
    else if (tot[1] == 0.0 && tot[2] == 0.0) st->done = 2;
  }
}

// p = r (first step after a start or restart) or p = r + beta (p - omega v).
__global__ void k_update_p_kernel(KrylovVecs k) {
  pdl_enter();
  k = instance(k);
  KState* st = k.st;
  if (st->done == 5 && st->it > st->maxit) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 4;
    return;
  }
  if (st->done == 5) {
    // Near-breakdown restart: a new pseudo-random shadow residual (the next seed of the same
    // generator), p = r, rho = <r^, r>.
    const unsigned long long seed = SHADOW_SEED + 0x2545F4914F6CDD1Dull * (unsigned long long)(st->shadow_restarts + 1);
    double acc[3] = {0.0, 0.0, 0.0};
    const int N = (int)k.N;
    GRID_STRIDE(e, N) {
      const double2 rh = shadow_value(seed, e), r = k.r[e];
      k.rhat[e] = rh;
      k.p[e] = r;
      if (k.p32) k.p32[e] = narrow(r);
      acc[0] = fma(rh.x, r.x, fma(rh.y, r.y, acc[0]));
      acc[1] = fma(rh.x, r.y, fma(-rh.y, r.x, acc[1]));
      acc[2] = fma(rh.x, rh.x, fma(rh.y, rh.y, acc[2]));
    }
    double tot[3];
    if (!grid_sum<3>(acc, k.partials, &st->ticket[KT_SHADOW], tot)) return;
    if (threadIdx.x == 0) {
      st->rho = make_double2(tot[0], tot[1]);
      st->rhat2 = tot[2];
      st->first = 0;
      st->shadow_restarts += 1;
      st->done = (tot[0] == 0.0 && tot[1] == 0.0) ? 2 : 0;
      if (st->done) st->iters_x2 = 2 * (st->it - 1);
    }
    return;
  }
  if (st->done) return;
  if (st->it > st->maxit) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->done = 4;
    return;
  }
  const int N = (int)k.N;
  const int first = st->first;
  const double2 beta = st->beta, omega = st->omega;
  GRID_STRIDE(e, N) {
    double2 r = k.r[e];
    double2 p;
    if (first) {
      p = r;
    } else {
      double2 q = d2axmy(k.p[e], omega, k.v[e]);
      p = d2axpy(r, beta, q);
    }
    k.p[e] = p;
    if (k.p32) k.p32[e] = narrow(p);
  }
}

// v = A y with <r^, v>; alpha = rho / <r^, v>.
template <class Y2>
__global__ void k_apply_rv_kernel(KrylovVecs k, const Y2* __restrict__ y) {
  pdl_enter();
  k = instance(k);
  y += blockIdx.z * k.sv;
  KState* st = k.st;
  if (st->done) return;
  double acc[2] = {0.0, 0.0};
  const int N = (int)k.N;
  for (NodeWalk it(k.n, gridDim.x * KB); it.e < N; it.next()) {
    const int e = it.e;
    double2 v = apply_at(y, k.kh, e, it.i, it.j, k.n, 0.0);
    k.v[e] = v;
    double2 rh = k.rhat[e];
    acc[0] = fma(rh.x, v.x, fma(rh.y, v.y, acc[0]));
    acc[1] = fma(rh.x, v.y, fma(-rh.y, v.x, acc[1]));
  }
  double tot[2];
  if (!grid_sum<2>(acc, k.partials, &st->ticket[KT_RV], tot)) return;
  if (threadIdx.x == 0) {
    double2 rv = make_double2(tot[0], tot[1]);
    st->rv = rv;
    if (!fin2(rv)) {
      st->done = 3;
    } else if (rv.x == 0.0 && rv.y == 0.0) {
      st->done = 2;
      st->iters_x2 = 2 * (st->it - 1);
    } else {
      st->alpha = d2div(st->rho, rv);
      st->alpha_x = st->alpha;  // x += alpha y is due (k_update_x, beside the next preconditioner application)
      st->xa = 1;
    }
  }
}

// s = r - alpha v with |s|^2; stop after the half step when |s| <= tol |b|.
__global__ void k_update_s_kernel(KrylovVecs k) {
  pdl_enter();
  k = instance(k);
  KState* st = k.st;
  if (st->done) return;
  double acc[1] = {0.0};
  const double2 alpha = st->alpha;
  const int N = (int)k.N;
  GRID_STRIDE(e, N) {
    double2 s = d2axmy(k.r[e], alpha, k.v[e]);
    k.s[e] = s;
    if (k.s32) k.s32[e] = narrow(s);
    acc[0] = fma(s.x, s.x, fma(s.y, s.y, acc[0]));
  }
  double tot[1];
  if (!grid_sum<1>(acc, k.partials, &st->ticket[KT_S], tot)) return;
  if (threadIdx.x == 0) {
    st->ss = tot[0];
    hist_push(st, k.hist, sqrt(tot[0] / st->bnorm2));
    if (!fin(tot[0])) {
      st->done = 3;
    } else if (tot[0] <= st->tol2) {
      st->half = 1;
      st->done = 1;
      st->iters_x2 = 2 * st->it - 1;
    }
  }
}

// t = A z with <t, s> and <t, t>; omega = <t, s> / <t, t>.
template <class Y2>
__global__ void k_apply_ts_kernel(KrylovVecs k, const Y2* __restrict__ z) {
  pdl_enter();
  k = instance(k);
  z += blockIdx.z * k.sv;
  KState* st = k.st;
  if (st->done) return;
  double acc[3] = {0.0, 0.0, 0.0};
  const int N = (int)k.N;
  for (NodeWalk it(k.n, gridDim.x * KB); it.e < N; it.next()) {
    const int e = it.e;
    double2 t = apply_at(z, k.kh, e, it.i, it.j, k.n, 0.0);
    k.t[e] = t;
    double2 s = k.s[e];
    acc[0] = fma(t.x, s.x, fma(t.y, s.y, acc[0]));
    acc[1] = fma(t.x, s.y, fma(-t.y, s.x, acc[1]));
    acc[2] = fma(t.x, t.x, fma(t.y, t.y, acc[2]));
  }
  double tot[3];
  if (!grid_sum<3>(acc, k.partials, &st->ticket[KT_TS], tot)) return;
  if (threadIdx.x == 0) {
    st->ts = make_double2(tot[0], tot[1]);
    st->tt = tot[2];
    if (!fin(tot[0]) || !fin(tot[1]) || !fin(tot[2])) {
      st->done = 3;
    } else if (tot[2] == 0.0) {
      st->done = 2;
      st->iters_x2 = 2 * (st->it - 1);
    } else {
      st->omega = make_double2(tot[0] / tot[2], tot[1] / tot[2]);
    }
  }
}

// r = s - omega t with <r^, r> and |r|^2; the next beta. This step's solution update (x += alpha y
// + omega z) is deferred to k_update_x.
__global__ void k_update_r_kernel(KrylovVecs k) {
  pdl_enter();
  k = instance(k);
  KState* st = k.st;
  if (st->done) return;
  double acc[3] = {0.0, 0.0, 0.0};
  const double2 alpha = st->alpha, omega = st->omega;
  const int N = (int)k.N;
  GRID_STRIDE(e, N) {
    double2 r = d2axmy(k.s[e], omega, k.t[e]);
    k.r[e] = r;
    double2 rh = k.rhat[e];
    acc[0] = fma(rh.x, r.x, fma(rh.y, r.y, acc[0]));
    acc[1] = fma(rh.x, r.y, fma(-rh.y, r.x, acc[1]));
    acc[2] = fma(r.x, r.x, fma(r.y, r.y, acc[2]));
  }
  double tot[3];
  if (!grid_sum<3>(acc, k.partials, &st->ticket[KT_XR], tot)) return;
  if (threadIdx.x == 0) {
    st->omega_x = omega;  // x += omega z is due (k_update_x, beside the next preconditioner application)
    st->xw = 1;
    st->rr = tot[2];
    hist_push(st, k.hist, sqrt(tot[2] / st->bnorm2));
    double2 rho_new = make_double2(tot[0], tot[1]);
    if (!fin(tot[0]) || !fin(tot[1]) || !fin(tot[2])) {
      st->done = 3;
    } else if (omega.x == 0.0 && omega.y == 0.0) {
      st->done = 2;
      st->iters_x2 = 2 * st->it;
    } else if (tot[2] <= st->tol2) {
      st->done = 1;
      st->iters_x2 = 2 * st->it;
    } else if (rho_new.x == 0.0 && rho_new.y == 0.0) {
      st->done = 2;
      st->iters_x2 = 2 * st->it;
    }
    if (!st->done) {  // here |r|^2 > tol2 > 0
      const double cos2 = (rho_new.x * rho_new.x + rho_new.y * rho_new.y) / (st->rhat2 * tot[2]);
      st->min_cos2 = fmin(st->min_cos2, cos2);
      const double step2 = (omega.x * omega.x + omega.y * omega.y) * st->tt / tot[2];
      if (cos2 < st->stall_cos2) st->min_step2 = fmin(st->min_step2, step2);
      if (cos2 < st->stall_cos2 && step2 < st->stall_step2 && st->shadow_restarts < st->max_shadow_restarts) {
        // <r^, r> has collapsed relative to |r^| |r| and the iteration no longer moves r: the
        // recurrences stall (alpha, omega -> 0) unless the shadow residual is renewed; the next
        // direction update restarts from r.
        st->done = 5;
        st->it += 1;
      }
    }
    if (!st->done) {
      st->rho_old = st->rho;
      st->rho = rho_new;
      st->beta = d2mul(d2div(rho_new, st->rho_old), d2div(alpha, omega));
      st->first = 0;
      st->it += 1;
    }
  }
}

// The deferred solution update, in two halves that keep the order of an immediate
// x += alpha y + omega z (two FMA-based complex updates per node, alpha y first), so the bits do
// not change: half A applies x += alpha y of the last step whose alpha was computed (KState::xa),
// half W x += omega z of the last full step (xw). Half A runs on a side branch beside the next
// step's first preconditioner application, which leaves x and y alone until its finest
// post-smoothing pass (which waits for it) writes y; half W beside the second one, likewise
// for z; after the last step both run once more, A first. One 128-thread block per SM with four
// nodes in flight per thread: few threads and registers, leaving the SMs to the V-cycle kernels.
constexpr int XB = 128;  // threads per block of k_update_x
template <class Y2, bool W>
__global__ void __launch_bounds__(XB, 8) k_update_x_kernel(KrylovVecs k, const Y2* __restrict__ yz) {
  pdl_enter();
  k = instance(k);
  yz += blockIdx.z * k.sv;
  KState* st = k.st;
  int* flag = W ? &st->xw : &st->xa;
  if (!*flag) return;
  const double2 c = W ? st->omega_x : st->alpha_x;
  const int N = (int)k.N, stride = gridDim.x * XB;
  int e = blockIdx.x * XB + threadIdx.x;
  for (; e + 3 * stride < N; e += 4 * stride) {
    double2 x[4];
    Y2 a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      x[q] = k.x[e + q * stride];
      a[q] = yz[e + q * stride];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) k.x[e + q * stride] = d2axpy(x[q], c, widen(a[q]));
  }
  for (; e < N; e += stride) k.x[e] = d2axpy(k.x[e], c, ldy(yz, e));
  // the last block to finish clears the flag (every block has read it by then)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket[W ? KT_XW : KT_XA], 1u);
    if (t == gridDim.x - 1) {
      *flag = 0;
      st->ticket[W ? KT_XW : KT_XA] = 0;
    }
  }
}

// One thread: count the iteration and set the WHILE node's condition (see LoopCtl).
__global__ void loop_control_kernel(LoopCtl c) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  const int cnt = ++*c.counter;
  bool running = false;
  int cap = 0;
  for (int p = 0; p < c.problems; ++p)
    for (int b = 0; b < c.batch[p]; ++b) {
      const KState& s = c.st[p][b];
      running = running || s.done == 0 || s.done == 5;
      cap = max(cap, s.maxit + 2);
    }
  cudaGraphSetConditional(c.handle, (running && cnt < cap) ? 1u : 0u);
}

// tr = h^2 b - A x and |tr|^2, to confirm a recurrence-converged iterate.
__global__ void k_true_residual_kernel(KrylovVecs k) {
  pdl_enter();
  k = instance(k);
  KState* st = k.st;
  double acc[1] = {0.0};
  const int N = (int)k.N;
  for (NodeWalk it(k.n, gridDim.x * KB); it.e < N; it.next()) {
    const int e = it.e;
    double2 ax = apply_at(k.x, k.kh, e, it.i, it.j, k.n, 0.0);
    double2 bv = k.b[e];
    double2 tr = make_double2(fma(bv.x, k.scale_b, -ax.x), fma(bv.y, k.scale_b, -ax.y));
    k.tr[e] = tr;
    acc[0] = fma(tr.x, tr.x, fma(tr.y, tr.y, acc[0]));
  }
  double tot[1];
  if (!grid_sum<1>(acc, k.partials, &st->ticket[KT_TRUE], tot)) return;
  if (threadIdx.x == 0) st->trr = tot[0];
}

// Restart from the true residual: r = tr, rho = <r^, r>, next step p = r.
__global__ void k_restart_kernel(KrylovVecs k) {
  pdl_enter();
  k = instance(k);
  KState* st = k.st;
  double acc[3] = {0.0, 0.0, 0.0};
  const int N = (int)k.N;
  GRID_STRIDE(e, N) {
    double2 r = k.tr[e];
    k.r[e] = r;
    double2 rh = k.rhat[e];
    acc[0] = fma(rh.x, r.x, fma(rh.y, r.y, acc[0]));
    acc[1] = fma(rh.x, r.y, fma(-rh.y, r.x, acc[1]));
    acc[2] = fma(r.x, r.x, fma(r.y, r.y, acc[2]));
  }
  double tot[3];
  if (!grid_sum<3>(acc, k.partials, &st->ticket[KT_RESTART], tot)) return;
  if (threadIdx.x == 0) {
    st->rho = make_double2(tot[0], tot[1]);
    st->rr = tot[2];
    st->first = 1;
    st->half = 0;
    st->done = 0;
    st->it += 1;
    if (tot[0] == 0.0 && tot[1] == 0.0) {
      st->done = 2;
      st->iters_x2 = 2 * (st->it - 1);
    }
  }
}

__global__ void apply_fp64_kernel(double2* v, const double2* u, const double* kh, int n, double beta,
                                  double out_scale) {
  pdl_enter();
  const int N = (n + 1) * (n + 1);
  for (NodeWalk it(n, gridDim.x * KB); it.e < N; it.next()) {
    const int e = it.e;
    double2 a = apply_at(u, kh, e, it.i, it.j, n, beta);
    v[e] = make_double2(a.x * out_scale, a.y * out_scale);
  }
}

}  // namespace

#define KGRID dim3(k.G, 1, k.batch)
#define KLAUNCH(name) pdl_launch(name, KGRID, KB, 0, s, k); return cudaGetLastError();

KrylovVecs instance_of(const KrylovVecs& k, int b) {
  KrylovVecs r = offset_instance(k, b);
  r.batch = 1;
  return r;
}

cudaError_t launch_k_init(const KrylovVecs& k, double tol, int maxit, int hist_cap, cudaStream_t s) {
  pdl_launch(k_init_kernel, KGRID, KB, 0, s, k, tol, maxit, hist_cap);
  return cudaGetLastError();
}
cudaError_t launch_k_update_p(const KrylovVecs& k, cudaStream_t s) { KLAUNCH(k_update_p_kernel) }
cudaError_t launch_k_apply_rv(const KrylovVecs& k, cudaStream_t s) {
  if (k.y32) pdl_launch(k_apply_rv_kernel<float2>, KGRID, KB, 0, s, k, k.y32);
  else pdl_launch(k_apply_rv_kernel<double2>, KGRID, KB, 0, s, k, k.y);
  return cudaGetLastError();
}
cudaError_t launch_k_update_s(const KrylovVecs& k, cudaStream_t s) { KLAUNCH(k_update_s_kernel) }
cudaError_t launch_k_apply_ts(const KrylovVecs& k, cudaStream_t s) {
  if (k.z32) pdl_launch(k_apply_ts_kernel<float2>, KGRID, KB, 0, s, k, k.z32);
  else pdl_launch(k_apply_ts_kernel<double2>, KGRID, KB, 0, s, k, k.z);
  return cudaGetLastError();
}
cudaError_t launch_k_update_r(const KrylovVecs& k, cudaStream_t s) { KLAUNCH(k_update_r_kernel) }
cudaError_t launch_k_update_x(const KrylovVecs& k, bool omega_half, cudaStream_t s) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || sms < 1) sms = 1;
  }
  const dim3 grid(sms, 1, k.batch);  // one block per SM: the V-cycle kernels beside it keep the rest
  if (k.y32) {
    if (omega_half) pdl_launch(k_update_x_kernel<float2, true>, grid, XB, 0, s, k, (const float2*)k.z32);
    else pdl_launch(k_update_x_kernel<float2, false>, grid, XB, 0, s, k, (const float2*)k.y32);
  } else {
    if (omega_half) pdl_launch(k_update_x_kernel<double2, true>, grid, XB, 0, s, k, (const double2*)k.z);
    else pdl_launch(k_update_x_kernel<double2, false>, grid, XB, 0, s, k, (const double2*)k.y);
  }
  return cudaGetLastError();
}
cudaError_t launch_k_true_residual(const KrylovVecs& k, cudaStream_t s) { KLAUNCH(k_true_residual_kernel) }
cudaError_t launch_loop_control(const LoopCtl& c, cudaStream_t s) {
  pdl_launch(loop_control_kernel, 1, 32, 0, s, c);
  return cudaGetLastError();
}
cudaError_t launch_k_restart(const KrylovVecs& k, cudaStream_t s) { KLAUNCH(k_restart_kernel) }

cudaError_t launch_apply_fp64(double2* v, const double2* u, const double* kh, int n, double beta, double out_scale,
                              cudaStream_t s) {
  long long N = (long long)(n + 1) * (n + 1);
  int G = (int)((N + KB - 1) / KB);
  if (G > 4096) G = 4096;
  pdl_launch(apply_fp64_kernel, G, KB, 0, s, v, u, kh, n, beta, out_scale);
  return cudaGetLastError();
}

}  // namespace hz
