// Register-streaming forms of the two fused Gauss-Seidel passes (FP32 form).
//
// The same arithmetic as the shared-memory tile kernels (Sec. 5: one red-black sweep from a zero
// guess, residual with the level's (B) operator and full weighting; bilinear correction and one
// sweep black first), laid out for the memory system instead of for shared memory. A warp owns a
// strip 64 nodes wide (lane L holds columns gx + 2L and gx + 2L + 1) and walks a segment of rows
// top to bottom, keeping the last four rows of u in registers: the red nodes of the newest row,
// the black nodes one row behind and the residual two rows behind are all final when computed,
// so every stage is a few register operations plus one or two lane shuffles for the horizontal
// neighbours. Input rows are loaded four rows ahead of use (16-byte loads per lane, a warp reads
// 512 contiguous bytes per row), so a warp keeps several kilobytes in flight without waiting,
// and no block ever synchronises.
//
// Boundaries: nodes outside the square are computed as copies of their mirror images (the loads
// reflect the row and column indices; a node's number of boundary sides is taken from its mirror
// image), which is the ghost elimination of the first-order Sommerfeld rows: the mirror copy
// equals the mirror node bit for bit because both are computed from the same values in the same
// order, so the boundary row sees 2 u_mirror exactly.
#include <cuda_runtime.h>

#include <stdint.h>

#include "hz_common.cuh"
#include "hz_internal.h"

namespace hz {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct L2c {  // a lane's two adjacent columns
  float2 a, b;
};

__device__ __forceinline__ int mirror_index(int i, int n) {
  i = i < 0 ? -i : i;
  i = i > n ? 2 * n - i : i;
  return i < 0 ? 0 : i;  // beyond one reflection: any node (such lanes never feed an output)
}
__device__ __forceinline__ float2 shfl_up2(float2 v) {
  return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
  return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return xr::cadd<float>(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return xr::csub<float>(a, b); }
__device__ __forceinline__ float2 scl2(float2 a, float s) { return xr::cscale<float>(a, s); }
__device__ __forceinline__ float2 diag(float k, int sides, float beta) { return xr::diag<float>(k, sides, beta); }
__device__ __forceinline__ float2 div2(float2 a, float2 d) { return xr::cdiv<float>(a, d); }
__device__ __forceinline__ float2 mul2(float2 d, float2 u) { return xr::cmul<float>(d, u); }
__device__ __forceinline__ int sides_of(int m, int n) { return (m == 0) + (m == n); }

// Row loads for a lane's pair of columns. EDGE strips reflect each column; elsewhere a pair is one
// 16-byte load when VEC (row starts 16-byte aligned), else two 8-byte loads.
template <bool EDGE, bool VEC>
__device__ __forceinline__ void load_pair(const float2* __restrict__ row, int c0, int m0, int m1, L2c& U) {
  if (EDGE) {
    U.a = __ldg(row + m0);
    U.b = __ldg(row + m1);
  } else if (VEC) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row + c0));
    U.a = make_float2(v.x, v.y);
    U.b = make_float2(v.z, v.w);
  } else {
    U.a = __ldg(row + c0);
    U.b = __ldg(row + c0 + 1);
  }
}
template <bool EDGE>
__device__ __forceinline__ float2 load_k(const float* __restrict__ krow, int c0, int m0, int m1) {
  if (EDGE) return make_float2(__ldg(krow + m0), __ldg(krow + m1));
  return __ldg(reinterpret_cast<const float2*>(krow + c0));
}
// Store a lane's pair where lo <= column <= hi (a lane stores both or, at the grid edge, one).
template <bool VEC>
__device__ __forceinline__ void store_pair(float2* __restrict__ row, int c0, int lo, int hi, const L2c& U) {
  const bool s0 = c0 >= lo && c0 <= hi, s1 = c0 + 1 >= lo && c0 + 1 <= hi;
  if (VEC && s0 && s1) {
    *reinterpret_cast<float4*>(row + c0) = make_float4(U.a.x, U.a.y, U.b.x, U.b.y);
  } else {
    if (s0) row[c0] = U.a;
    if (s1) row[c0 + 1] = U.b;
  }
}

// ------------------------------------------------------------------ smooth + residual + restrict
// Strip: columns gx .. gx + 63 with gx = 58 s - 4; the strip's outputs are columns gx + 4 ..
// gx + 61 (u) and coarse columns gx/2 + 2 .. gx/2 + 30. Segment: output rows y0 .. row_end - 1;
// loaded rows y0 - 3 .. row_end + 2, stage t handling loaded row t (global y0 - 3 + t):
//   red at row t, black at row t-1 (u of row t-1 final, stored), residual at row t-2 and its
//   full-weighting accumulation (coarse row J completes at fine row 2J + 1).
constexpr int SR_W = 58;

struct SRState {
  L2c F[8];
  float2 K[8];
  L2c U[4];
  float2 hS, hC;  // full-weighting row sums of rows 2J - 1 and 2J
};

struct SRArgs {
  float2* u;
  int pu;
  float2* fc;
  int pc;
  const float2* f;
  int pf;
  const float* kh;
  int pk;
  int n;
  float bA, bB;
};

template <int Q, bool EDGE, bool VF>
__device__ __forceinline__ void sr_stage(SRState& S, const SRArgs& A, int t, int T, int y0, int row_end, int gx,
                                         int c0, int m0, int m1, int sc0, int sc1) {
  if (t >= T) return;
  const int L = threadIdx.x;
  // prefetch row t + 4
  if (t + 4 < T) {
    const int mj = mirror_index(y0 + 1 + t, A.n);
    load_pair<EDGE, VF>(A.f + (long long)mj * A.pf, c0, m0, m1, S.F[(Q + 4) & 7]);
    S.K[(Q + 4) & 7] = load_k<EDGE>(A.kh + (long long)mj * A.pk, c0, m0, m1);
  }
  // global row y0 - 3 + t has the parity of t + 1: red is column 0 of the pair on odd t
  constexpr int er = (Q & 1) ? 0 : 1;
  const int rs0 = sides_of(mirror_index(y0 - 3 + t, A.n), A.n);
  {  // red at row t (zero guess)
    L2c& U = S.U[Q & 3];
    if (er == 0)
      U.a = div2(S.F[Q].a, diag(S.K[Q].x, sc0 + rs0, A.bA));
    else
      U.b = div2(S.F[Q].b, diag(S.K[Q].y, sc1 + rs0, A.bA));
  }
  if (t >= 1) {  // black at row t-1, column er
    constexpr int q1 = (Q + 7) & 7, u1 = (Q + 3) & 3, u2 = (Q + 2) & 3, u0 = Q & 3;
    const int rs1 = sides_of(mirror_index(y0 - 4 + t, A.n), A.n);
    L2c& U = S.U[u1];
    if (er == 1) {
      const float2 right = shfl_down2(U.a);
      const float2 nb = add2(add2(U.a, right), add2(S.U[u2].b, S.U[u0].b));
      U.b = div2(sub2(S.F[q1].b, nb), diag(S.K[q1].y, sc1 + rs1, A.bA));
    } else {
      const float2 left = shfl_up2(U.b);
      const float2 nb = add2(add2(left, U.b), add2(S.U[u2].a, S.U[u0].a));
      U.a = div2(sub2(S.F[q1].a, nb), diag(S.K[q1].x, sc0 + rs1, A.bA));
    }
    const int jo = y0 - 4 + t;
    if (jo >= y0 && jo < row_end) store_pair<true>(A.u + (long long)jo * A.pu, c0, gx + 4, min(gx + 61, A.n), U);
  }
  if (t >= 2) {  // residual f - B u at row t-2 and its full-weighting accumulation
    constexpr int q2 = (Q + 6) & 7, u1 = (Q + 3) & 3, u2 = (Q + 2) & 3, u3 = (Q + 1) & 3;
    const int rs2 = sides_of(mirror_index(y0 - 5 + t, A.n), A.n);
    const L2c& U = S.U[u2];
    const float2 left = shfl_up2(U.b), right = shfl_down2(U.a);
    L2c R;
    R.a = sub2(S.F[q2].a, add2(mul2(diag(S.K[q2].x, sc0 + rs2, A.bB), U.a),
                               add2(add2(left, U.b), add2(S.U[u3].a, S.U[u1].a))));
    R.b = sub2(S.F[q2].b, add2(mul2(diag(S.K[q2].y, sc1 + rs2, A.bB), U.b),
                               add2(add2(U.a, right), add2(S.U[u3].b, S.U[u1].b))));
    // full weighting: the row sum (w + e) + 2 c at this lane's coarse column (2I = c0), then
    // across rows. Row y0 - 5 + t is even (2J) on odd t, odd (2J + 1) on even t.
    const float2 h = xr::fw3<float>(shfl_up2(R.b), R.a, R.b);
    if (Q & 1) {
      S.hC = h;
    } else {
      const int j2 = y0 - 6 + t;  // = 2J
      if (j2 >= y0 && j2 < row_end) {
        const int I = (gx >> 1) + L;
        if (L >= 2 && L <= 30 && I <= (A.n >> 1))
          A.fc[(long long)(j2 >> 1) * A.pc + I] = scl2(xr::fw3<float>(S.hS, S.hC, h), 0.25f);
      }
      S.hS = h;
    }
  }
}

template <bool EDGE, bool VF>
__device__ __forceinline__ void sr_run(const SRArgs& A, int gx, int y0, int row_end) {
  const int L = threadIdx.x;
  const int c0 = gx + 2 * L;
  const int m0 = mirror_index(c0, A.n), m1 = mirror_index(c0 + 1, A.n);
  const int sc0 = sides_of(m0, A.n), sc1 = sides_of(m1, A.n);
  const int T = row_end - y0 + 6;
  SRState S;
#pragma unroll
  for (int q = 0; q < 4; ++q) S.U[q].a = S.U[q].b = make_float2(0.f, 0.f);
  S.hS = S.hC = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < T) {
      const int mj = mirror_index(y0 - 3 + q, A.n);
      load_pair<EDGE, VF>(A.f + (long long)mj * A.pf, c0, m0, m1, S.F[q]);
      S.K[q] = load_k<EDGE>(A.kh + (long long)mj * A.pk, c0, m0, m1);
    }
  }
  for (int t0 = 0; t0 < T; t0 += 8) {
    sr_stage<0, EDGE, VF>(S, A, t0 + 0, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<1, EDGE, VF>(S, A, t0 + 1, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<2, EDGE, VF>(S, A, t0 + 2, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<3, EDGE, VF>(S, A, t0 + 3, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<4, EDGE, VF>(S, A, t0 + 4, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<5, EDGE, VF>(S, A, t0 + 5, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<6, EDGE, VF>(S, A, t0 + 6, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
    sr_stage<7, EDGE, VF>(S, A, t0 + 7, T, y0, row_end, gx, c0, m0, m1, sc0, sc1);
  }
}

template <bool VF>
__global__ void __launch_bounds__(128) smooth_restrict_stream_kernel(SRArgs A, int strips, int seg_rows,
                                                                      const int* __restrict__ stop, Inst bi) {
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * blockDim.y + threadIdx.y;
  if (strip >= strips) return;  // whole warp
  A.u += blockIdx.z * bi.su;
  A.fc += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * SR_W - 4;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    sr_run<false, VF>(A, gx, y0, row_end);
  else
    sr_run<true, VF>(A, gx, y0, row_end);
}

// ------------------------------------------------------------------ prolong + post-smooth
// Strip: columns gx .. gx + 63 with gx = 58 s - 2; outputs gx + 2 .. gx + 59 (v = u_pre + P e_c
// is valid on gx .. gx + 62: the odd column of the last lane would need the next lane's coarse
// value; black nodes on gx + 1 .. gx + 61; red on gx + 2 .. gx + 60). Loaded rows y0 - 2 ..
// row_end + 1, plus the coarse row under row_end + 2 when row_end + 1 is odd; stage t: v at row t,
// black at row t-1 (from v), red at row t-2 (from the updated black nodes), row t-2 stored.
constexpr int PS_W = 58;

struct PSState {
  L2c F[8];
  float2 K[8];
  L2c V[8];      // u_pre rows, loaded ahead
  float2 E[4];   // coarse e at this lane's coarse column, one slot per even fine row
  L2c U[4];
};

struct PSArgs {
  float2* out;
  int po;
  const float2* upre;
  int pu;
  const float2* ec;
  int pc;
  const float2* f;
  int pf;
  const float* kh;
  int pk;
  int n;
  float bA;
};

// Loads of loaded row t (< T) and, on even rows, of the coarse row under it (also for t == T,
// which the odd row T - 1 interpolates from).
template <bool EDGE, bool V>
__device__ __forceinline__ void ps_load(PSState& S, const PSArgs& A, int q, int t, int T, int y0, int c0, int m0,
                                        int m1, int ci) {
  const int j = y0 - 2 + t;
  if (t < T) {
    const int mj = mirror_index(j, A.n);
    load_pair<EDGE, V>(A.f + (long long)mj * A.pf, c0, m0, m1, S.F[q & 7]);
    S.K[q & 7] = load_k<EDGE>(A.kh + (long long)mj * A.pk, c0, m0, m1);
    load_pair<EDGE, true>(A.upre + (long long)mj * A.pu, c0, m0, m1, S.V[q & 7]);
  }
  if (!(j & 1)) S.E[(q >> 1) & 3] = __ldg(A.ec + (long long)mirror_index(j >> 1, A.n >> 1) * A.pc + ci);
}

template <int Q, bool EDGE, bool V>
__device__ __forceinline__ void ps_stage(PSState& S, const PSArgs& A, int t, int T, int y0, int row_end, int gx,
                                         int c0, int m0, int m1, int ci, int sc0, int sc1) {
  if (t >= T) return;
  if (t + 4 <= T) ps_load<EDGE, V>(S, A, Q + 4, t + 4, T, y0, c0, m0, m1, ci);
  // global row y0 - 2 + t has the parity of t: red is column 0 of the pair on even t
  constexpr int er = (Q & 1) ? 1 : 0;
  {  // v = u_pre + P e at row t
    L2c& U = S.U[Q & 3];
    const L2c& Up = S.V[Q];
    if (Q & 1) {
      const float2 ev = add2(S.E[((Q - 1) >> 1) & 3], S.E[((Q + 1) >> 1) & 3]);
      const float2 evn = shfl_down2(ev);
      U.a = add2(Up.a, scl2(ev, 0.5f));
      U.b = add2(Up.b, scl2(add2(ev, evn), 0.25f));
    } else {
      const float2 e = S.E[(Q >> 1) & 3];
      const float2 en = shfl_down2(e);
      U.a = add2(Up.a, e);
      U.b = add2(Up.b, scl2(add2(e, en), 0.5f));
    }
  }
  if (t >= 1) {  // black at row t-1, column er (its vertical neighbours are red v nodes)
    constexpr int q1 = (Q + 7) & 7, u1 = (Q + 3) & 3, u2 = (Q + 2) & 3, u0 = Q & 3;
    const int rs1 = sides_of(mirror_index(y0 - 3 + t, A.n), A.n);
    L2c& U = S.U[u1];
    if (er == 1) {
      const float2 right = shfl_down2(U.a);
      const float2 nb = add2(add2(U.a, right), add2(S.U[u2].b, S.U[u0].b));
      U.b = div2(sub2(S.F[q1].b, nb), diag(S.K[q1].y, sc1 + rs1, A.bA));
    } else {
      const float2 left = shfl_up2(U.b);
      const float2 nb = add2(add2(left, U.b), add2(S.U[u2].a, S.U[u0].a));
      U.a = div2(sub2(S.F[q1].a, nb), diag(S.K[q1].x, sc0 + rs1, A.bA));
    }
  }
  if (t >= 2) {  // red at row t-2, column er (its neighbours are updated black nodes)
    constexpr int q2 = (Q + 6) & 7, u1 = (Q + 3) & 3, u2 = (Q + 2) & 3, u3 = (Q + 1) & 3;
    const int rs2 = sides_of(mirror_index(y0 - 4 + t, A.n), A.n);
    L2c& U = S.U[u2];
    if (er == 0) {
      const float2 left = shfl_up2(U.b);
      const float2 nb = add2(add2(left, U.b), add2(S.U[u3].a, S.U[u1].a));
      U.a = div2(sub2(S.F[q2].a, nb), diag(S.K[q2].x, sc0 + rs2, A.bA));
    } else {
      const float2 right = shfl_down2(U.a);
      const float2 nb = add2(add2(U.a, right), add2(S.U[u3].b, S.U[u1].b));
      U.b = div2(sub2(S.F[q2].b, nb), diag(S.K[q2].y, sc1 + rs2, A.bA));
    }
    const int jo = y0 - 4 + t;
    if (jo >= y0 && jo < row_end) store_pair<V>(A.out + (long long)jo * A.po, c0, max(gx + 2, 0), min(gx + 59, A.n), U);
  }
}

template <bool EDGE, bool V>
__device__ __forceinline__ void ps_run(const PSArgs& A, int gx, int y0, int row_end) {
  const int L = threadIdx.x;
  const int c0 = gx + 2 * L;
  const int m0 = mirror_index(c0, A.n), m1 = mirror_index(c0 + 1, A.n);
  const int ci = mirror_index(c0 >> 1, A.n >> 1);  // this lane's coarse column
  const int sc0 = sides_of(m0, A.n), sc1 = sides_of(m1, A.n);
  const int T = row_end - y0 + 4;
  PSState S;
#pragma unroll
  for (int q = 0; q < 4; ++q) S.U[q].a = S.U[q].b = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q <= T) ps_load<EDGE, V>(S, A, q, q, T, y0, c0, m0, m1, ci);
  for (int t0 = 0; t0 < T; t0 += 8) {
    ps_stage<0, EDGE, V>(S, A, t0 + 0, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<1, EDGE, V>(S, A, t0 + 1, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<2, EDGE, V>(S, A, t0 + 2, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<3, EDGE, V>(S, A, t0 + 3, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<4, EDGE, V>(S, A, t0 + 4, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<5, EDGE, V>(S, A, t0 + 5, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<6, EDGE, V>(S, A, t0 + 6, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
    ps_stage<7, EDGE, V>(S, A, t0 + 7, T, y0, row_end, gx, c0, m0, m1, ci, sc0, sc1);
  }
}

template <bool V>
__global__ void __launch_bounds__(128) prolong_smooth_stream_kernel(PSArgs A, int strips, int seg_rows,
                                                                     const int* __restrict__ stop, Inst bi) {
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * blockDim.y + threadIdx.y;
  if (strip >= strips) return;
  A.out += blockIdx.z * bi.so;
  A.upre += blockIdx.z * bi.su;
  A.ec += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * PS_W - 2;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    ps_run<false, V>(A, gx, y0, row_end);
  else
    ps_run<true, V>(A, gx, y0, row_end);
}

constexpr int WPB = 4;  // warps (strips) per block

bool aligned16(const void* p, long long pitch, long long stride) {
  return ((uintptr_t)p & 15) == 0 && !(pitch & 1) && !(stride & 1);
}

}  // namespace

cudaError_t launch_smooth_restrict_stream(void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                          int pk, int n, double bA, double bB, int seg_rows, const int* stop,
                                          cudaStream_t s, const Inst& bi) {
  if (seg_rows < 2 || (seg_rows & 1) || n < 4 || !aligned16(u, pu, bi.su) || !aligned16(kh, pk, 0))
    return cudaErrorInvalidValue;
  SRArgs A{(float2*)u, pu, (float2*)fc, pc, (const float2*)f, pf, (const float*)kh, pk, n, (float)bA, (float)bB};
  const int strips = (n + 1 + SR_W - 1) / SR_W, segs = (n + 1 + seg_rows - 1) / seg_rows;
  dim3 grid((strips + WPB - 1) / WPB, segs, bi.count);
  if (aligned16(f, pf, bi.sf))
    smooth_restrict_stream_kernel<true><<<grid, dim3(32, WPB), 0, s>>>(A, strips, seg_rows, stop, bi);
  else
    smooth_restrict_stream_kernel<false><<<grid, dim3(32, WPB), 0, s>>>(A, strips, seg_rows, stop, bi);
  return cudaGetLastError();
}

cudaError_t launch_prolong_smooth_stream(void* out, int po, const void* upre, int pu, const void* ec, int pc,
                                         const void* f, int pf, const void* kh, int pk, int n, double bA, int seg_rows,
                                         const int* stop, cudaStream_t s, const Inst& bi) {
  if (seg_rows < 2 || (seg_rows & 1) || n < 4 || !aligned16(upre, pu, bi.su) || !aligned16(kh, pk, 0))
    return cudaErrorInvalidValue;
  PSArgs A{(float2*)out, po, (const float2*)upre, pu, (const float2*)ec, pc, (const float2*)f, pf,
           (const float*)kh, pk, n, (float)bA};
  const int strips = (n + 1 + PS_W - 1) / PS_W, segs = (n + 1 + seg_rows - 1) / seg_rows;
  dim3 grid((strips + WPB - 1) / WPB, segs, bi.count);
  if (aligned16(f, pf, bi.sf) && aligned16(out, po, bi.so))
    prolong_smooth_stream_kernel<true><<<grid, dim3(32, WPB), 0, s>>>(A, strips, seg_rows, stop, bi);
  else
    prolong_smooth_stream_kernel<false><<<grid, dim3(32, WPB), 0, s>>>(A, strips, seg_rows, stop, bi);
  return cudaGetLastError();
}

}  // namespace hz
