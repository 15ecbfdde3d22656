// Register-streaming forms of the two fused Gauss-Seidel passes (FP32 form).
//
// The same arithmetic as the shared-memory tile kernels (Sec. 5: one red-black sweep from a zero
// guess, residual with the level's (B) operator and full weighting; bilinear correction and one
// sweep black first), laid out for the memory system instead of for shared memory. A warp owns a
// strip 64 nodes wide (lane L holds columns gx + 2L and gx + 2L + 1) and walks a segment of rows
// top to bottom, keeping the last four rows of u in registers: the red nodes of the newest row,
// the black nodes one row behind and the residual two rows behind are all final when computed,
// so every stage is a few register operations plus lane shuffles for the horizontal neighbours.
//
// Input rows arrive through a ring of R row slots in shared memory that each lane fills for its
// own columns with cp.async, several rows ahead of use: the copies hold no registers, so a warp
// keeps kilobytes in flight, and since a lane reads back only what it copied itself,
// cp.async.wait_group orders everything and no barrier or shared flag is needed. A slot is
// refilled at the end of the stage that consumed the registers loaded from it, so the refill
// cannot overtake the read.
//
// Boundaries: nodes outside the square are computed as copies of their mirror images (the copies
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
constexpr int WPB = 4;  // warps (strips) per block

struct L2c {  // a lane's two adjacent columns
  float2 a, b;
};

__device__ __forceinline__ int mirror_index(int i, int n) {
  i = i < 0 ? -i : i;
  i = i > n ? 2 * n - i : i;
  return i < 0 ? 0 : i;  // beyond one reflection: any node (such lanes never feed an output)
}
// Twice the boundary sides of row (or column) j, mirror images included (j in [-n, 2n]; n >= 1).
__device__ __forceinline__ float sides2(int j, int n) { return (j == 0 || j == n) ? 2.0f : 0.0f; }

__device__ __forceinline__ float2 shfl_up2(float2 v) {
  return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down2(float2 v) {
  return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return xr::cadd<float>(a, b); }
__device__ __forceinline__ float2 scl2(float2 a, float s) { return xr::cscale<float>(a, s); }
__device__ __forceinline__ float2 diag(float k, float two_sides, float beta) { return xr::diag2<float>(k, two_sides, beta); }

// ------------------------------------------------------------------ per-lane async copies
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp4(unsigned dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A lane's pair of complex values from `row` into 16 bytes at dst: one 16-byte copy when the pair
// is contiguous and aligned (VEC, interior strips), else two 8-byte copies (mirrored columns).
template <bool EDGE, bool VEC>
__device__ __forceinline__ void copy_pair(unsigned dst, const float2* row, int c0, int m0, int m1) {
  if (!EDGE && VEC) {
    cp16(dst, row + c0);
  } else {
    cp8(dst, row + (EDGE ? m0 : c0));
    cp8(dst + 8, row + (EDGE ? m1 : c0 + 1));
  }
}
template <bool EDGE>
__device__ __forceinline__ void copy_kpair(unsigned dst, const float* row, int c0, int m0, int m1) {
  if (!EDGE) {
    cp8(dst, row + c0);
  } else {
    cp4(dst, row + m0);
    cp4(dst + 4, row + m1);
  }
}
__device__ __forceinline__ L2c lds_pair(const unsigned char* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  L2c r;
  r.a = make_float2(v.x, v.y);
  r.b = make_float2(v.z, v.w);
  return r;
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

// Four-row window after two stages: slot k takes the row of slot k + 2 (mod 4), so the stage code
// written for slots 0 and 1 serves every pair of rows.
template <class X>
__device__ __forceinline__ void rotate2(X (&w)[4]) {
  const X a = w[0], b = w[1];
  w[0] = w[2];
  w[1] = w[3];
  w[2] = a;
  w[3] = b;
}

struct Lane {  // per-lane constants of a strip
  int c0, m0, m1;
  float sc0, sc1;  // twice the boundary sides of the two columns
};
__device__ __forceinline__ Lane lane_of(int gx, int n) {
  Lane q;
  q.c0 = gx + 2 * (int)threadIdx.x;
  q.m0 = mirror_index(q.c0, n);
  q.m1 = mirror_index(q.c0 + 1, n);
  q.sc0 = sides2(q.c0, n);
  q.sc1 = sides2(q.c0 + 1, n);
  return q;
}

// ------------------------------------------------------------------ smooth + residual + restrict
// Strip: columns gx .. gx + 63 with gx = 58 s - 4; the strip's outputs are columns gx + 4 ..
// gx + 61 (u) and coarse columns gx/2 + 2 .. gx/2 + 30. Segment: output rows y0 .. row_end - 1;
// loaded rows y0 - 3 .. row_end + 2, stage t handling loaded row t (global y0 - 3 + t):
//   red at row t, black at row t-1 (u of row t-1 final, stored), residual at row t-2 and its
//   full-weighting row sum (coarse row J completes at fine row 2J + 1).
constexpr int SR_W = 58;
constexpr int SR_R = 8;            // row slots per warp
constexpr int SR_SLOT = 32 * 24;   // bytes per slot: f pairs (16 B per lane), then k pairs (8 B)

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

struct SRState {
  L2c F[4];
  float2 K[4];
  L2c U[4];
  float2 hS, hC;  // full-weighting row sums of rows 2J - 1 and 2J
};

template <bool EDGE, bool VF>
__device__ __forceinline__ void sr_issue(unsigned char* ring, const SRArgs& A, int t, int T, int y0, const Lane& q) {
  if (t < T) {
    const int mj = mirror_index(y0 - 3 + t, A.n);
    unsigned char* slot = ring + (t % SR_R) * SR_SLOT;
    copy_pair<EDGE, VF>(smem_addr(slot + 16 * threadIdx.x), A.f + (long long)mj * A.pf, q.c0, q.m0, q.m1);
    copy_kpair<EDGE>(smem_addr(slot + 512 + 8 * threadIdx.x), A.kh + (long long)mj * A.pk, q.c0, q.m0, q.m1);
  }
  cp_commit();  // one group per row index, empty past the segment, so the wait count stays fixed
}

template <int Q, bool EDGE, bool VF>
__device__ __forceinline__ void sr_stage(SRState& S, unsigned char* ring, const SRArgs& A, int t, int T, int y0,
                                         int row_end, int gx, const Lane& q) {
  if (t >= T) return;
  cp_wait<SR_R - 2>();  // rows up to t have landed (t + R - 1 groups committed)
  {
    const unsigned char* slot = ring + (t % SR_R) * SR_SLOT;
    S.F[Q] = lds_pair(slot + 16 * threadIdx.x);
    S.K[Q] = *reinterpret_cast<const float2*>(slot + 512 + 8 * threadIdx.x);
  }
  // global row y0 - 3 + t has the parity of t + 1: red is column 0 of the pair on odd t
  constexpr int er = (Q & 1) ? 0 : 1;
  const int j0 = y0 - 3 + t;
  {  // red at row t (zero guess)
    L2c& U = S.U[Q];
    const float rs = sides2(j0, A.n);
    if (er == 0)
      U.a = xr::cdiv<float>(S.F[Q].a, diag(S.K[Q].x, q.sc0 + rs, A.bA));
    else
      U.b = xr::cdiv<float>(S.F[Q].b, diag(S.K[Q].y, q.sc1 + rs, A.bA));
  }
  if (t >= 1) {  // black at row t-1, column er
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3;
    const float rs = sides2(j0 - 1, A.n);
    L2c& U = S.U[q1];
    if (er == 1) {
      const float2 nb = xr::nb4<float>(U.a, shfl_down2(U.a), S.U[q2].b, S.U[Q].b);
      U.b = xr::gs<float>(S.F[q1].b, nb, diag(S.K[q1].y, q.sc1 + rs, A.bA));
    } else {
      const float2 nb = xr::nb4<float>(shfl_up2(U.b), U.b, S.U[q2].a, S.U[Q].a);
      U.a = xr::gs<float>(S.F[q1].a, nb, diag(S.K[q1].x, q.sc0 + rs, A.bA));
    }
    const int jo = j0 - 1;
    if (jo >= y0 && jo < row_end) store_pair<true>(A.u + (long long)jo * A.pu, q.c0, gx + 4, min(gx + 61, A.n), U);
  }
  if (t >= 2) {  // residual f - B u at row t-2 and its full-weighting row sum
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3, q3 = (Q + 1) & 3;
    const float rs = sides2(j0 - 2, A.n);
    const L2c& U = S.U[q2];
    L2c R;
    R.a = xr::resid<float>(S.F[q2].a, U.a, xr::nb4<float>(shfl_up2(U.b), U.b, S.U[q3].a, S.U[q1].a),
                           diag(S.K[q2].x, q.sc0 + rs, A.bB));
    R.b = xr::resid<float>(S.F[q2].b, U.b, xr::nb4<float>(U.a, shfl_down2(U.a), S.U[q3].b, S.U[q1].b),
                           diag(S.K[q2].y, q.sc1 + rs, A.bB));
    // the row sum (w + e) + 2 c at this lane's coarse column (2I = c0), then across rows; row
    // j0 - 2 is even (2J) on odd t, odd (2J + 1) on even t
    const float2 h = xr::fw3<float>(shfl_up2(R.b), R.a, R.b);
    if (Q & 1) {
      S.hC = h;
    } else {
      const int j2 = j0 - 3;  // = 2J
      if (j2 >= y0 && j2 < row_end) {
        const int L = threadIdx.x, I = (gx >> 1) + L;
        if (L >= 2 && L <= 30 && I <= (A.n >> 1))
          A.fc[(long long)(j2 >> 1) * A.pc + I] = scl2(xr::fw3<float>(S.hS, S.hC, h), 0.25f);
      }
      S.hS = h;
    }
  }
  // refill the slot of row t - 1, whose registers the black update above has consumed
  sr_issue<EDGE, VF>(ring, A, t + SR_R - 1, T, y0, q);
}

template <bool EDGE, bool VF>
__device__ __forceinline__ void sr_run(unsigned char* ring, const SRArgs& A, int gx, int y0, int row_end) {
  const Lane q = lane_of(gx, A.n);
  const int T = row_end - y0 + 6;
  SRState S;
#pragma unroll
  for (int k = 0; k < 4; ++k) S.U[k].a = S.U[k].b = make_float2(0.f, 0.f);
  S.hS = S.hC = make_float2(0.f, 0.f);
  for (int t = 0; t < SR_R - 1; ++t) sr_issue<EDGE, VF>(ring, A, t, T, y0, q);
  // two stages of code per iteration (a small loop body keeps the instruction cache warm when
  // few warps run); the four-row windows rotate by two rows between iterations
#pragma unroll 1
  for (int t0 = 0; t0 < T; t0 += 2) {
    sr_stage<0, EDGE, VF>(S, ring, A, t0 + 0, T, y0, row_end, gx, q);
    sr_stage<1, EDGE, VF>(S, ring, A, t0 + 1, T, y0, row_end, gx, q);
    rotate2(S.U);
    rotate2(S.F);
    rotate2(S.K);
  }
  cp_wait<0>();
}

template <bool VF>
__global__ void __launch_bounds__(32 * WPB) smooth_restrict_stream_kernel(SRArgs A, int strips, int seg_rows,
                                                                           const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * WPB + threadIdx.y;
  if (strip >= strips) return;  // whole warp
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ring = smem + threadIdx.y * SR_R * SR_SLOT;
  A.u += blockIdx.z * bi.su;
  A.fc += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * SR_W - 4;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    sr_run<false, VF>(ring, A, gx, y0, row_end);
  else
    sr_run<true, VF>(ring, A, gx, y0, row_end);
}

// ------------------------------------------------------------------ prolong + post-smooth
// Strip: columns gx .. gx + 63 with gx = 58 s - 2; outputs gx + 2 .. gx + 59 (v = u_pre + P e_c
// is valid on gx .. gx + 62: the odd column of the last lane would need the next lane's coarse
// value; black nodes on gx + 1 .. gx + 61; red on gx + 2 .. gx + 60). Loaded rows y0 - 2 ..
// row_end + 1, plus the coarse row under row_end + 2 when row_end + 1 is odd; stage t: v at row t,
// black at row t-1 (from v), red at row t-2 (from the updated black nodes), row t-2 stored.
constexpr int PS_W = 58;
constexpr int PS_R = 8;            // row slots per warp
constexpr int PS_SLOT = 32 * 48;   // f pairs (16 B per lane), u_pre pairs (16), k pairs (8), coarse e (8)

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

struct PSState {
  L2c F[4];
  float2 K[4];
  L2c U[4];
  float2 Ee;  // coarse e under the last even row
};

// Copies of loaded row t (< T) and, on even rows, of the coarse row under it (also for t == T,
// which the odd row T - 1 interpolates from).
template <bool EDGE, bool V>
__device__ __forceinline__ void ps_issue(unsigned char* ring, const PSArgs& A, int t, int T, int y0, const Lane& q,
                                         int ci) {
  if (t <= T) {
    const int j = y0 - 2 + t;
    unsigned char* slot = ring + (t % PS_R) * PS_SLOT;
    if (t < T) {
      const int mj = mirror_index(j, A.n);
      copy_pair<EDGE, V>(smem_addr(slot + 16 * threadIdx.x), A.f + (long long)mj * A.pf, q.c0, q.m0, q.m1);
      copy_pair<EDGE, true>(smem_addr(slot + 512 + 16 * threadIdx.x), A.upre + (long long)mj * A.pu, q.c0, q.m0,
                            q.m1);
      copy_kpair<EDGE>(smem_addr(slot + 1024 + 8 * threadIdx.x), A.kh + (long long)mj * A.pk, q.c0, q.m0, q.m1);
    }
    if (!(j & 1))
      cp8(smem_addr(slot + 1280 + 8 * threadIdx.x), A.ec + (long long)mirror_index(j >> 1, A.n >> 1) * A.pc + ci);
  }
  cp_commit();
}

template <int Q, bool EDGE, bool V>
__device__ __forceinline__ void ps_stage(PSState& S, unsigned char* ring, const PSArgs& A, int t, int T, int y0,
                                         int row_end, int gx, const Lane& q, int ci) {
  if (t >= T) return;
  cp_wait<PS_R - 3>();  // rows up to t + 1 have landed (t + R - 1 groups committed)
  const unsigned char* slot = ring + (t % PS_R) * PS_SLOT;
  S.F[Q] = lds_pair(slot + 16 * threadIdx.x);
  S.K[Q] = *reinterpret_cast<const float2*>(slot + 1024 + 8 * threadIdx.x);
  // global row y0 - 2 + t has the parity of t: red is column 0 of the pair on even t
  constexpr int er = (Q & 1) ? 1 : 0;
  const int j0 = y0 - 2 + t;
  {  // v = u_pre + P e at row t
    const L2c up = lds_pair(slot + 512 + 16 * threadIdx.x);
    L2c& U = S.U[Q];
    if (Q & 1) {
      const unsigned char* next = ring + ((t + 1) % PS_R) * PS_SLOT;
      const float2 ev = add2(S.Ee, *reinterpret_cast<const float2*>(next + 1280 + 8 * threadIdx.x));
      U.a = add2(up.a, scl2(ev, 0.5f));
      U.b = add2(up.b, scl2(add2(ev, shfl_down2(ev)), 0.25f));
    } else {
      S.Ee = *reinterpret_cast<const float2*>(slot + 1280 + 8 * threadIdx.x);
      U.a = add2(up.a, S.Ee);
      U.b = add2(up.b, scl2(add2(S.Ee, shfl_down2(S.Ee)), 0.5f));
    }
  }
  if (t >= 1) {  // black at row t-1, column er (its vertical neighbours are red v nodes)
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3;
    const float rs = sides2(j0 - 1, A.n);
    L2c& U = S.U[q1];
    if (er == 1) {
      const float2 nb = xr::nb4<float>(U.a, shfl_down2(U.a), S.U[q2].b, S.U[Q].b);
      U.b = xr::gs<float>(S.F[q1].b, nb, diag(S.K[q1].y, q.sc1 + rs, A.bA));
    } else {
      const float2 nb = xr::nb4<float>(shfl_up2(U.b), U.b, S.U[q2].a, S.U[Q].a);
      U.a = xr::gs<float>(S.F[q1].a, nb, diag(S.K[q1].x, q.sc0 + rs, A.bA));
    }
  }
  if (t >= 2) {  // red at row t-2, column er (its neighbours are updated black nodes)
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3, q3 = (Q + 1) & 3;
    const float rs = sides2(j0 - 2, A.n);
    L2c& U = S.U[q2];
    if (er == 0) {
      const float2 nb = xr::nb4<float>(shfl_up2(U.b), U.b, S.U[q3].a, S.U[q1].a);
      U.a = xr::gs<float>(S.F[q2].a, nb, diag(S.K[q2].x, q.sc0 + rs, A.bA));
    } else {
      const float2 nb = xr::nb4<float>(U.a, shfl_down2(U.a), S.U[q3].b, S.U[q1].b);
      U.b = xr::gs<float>(S.F[q2].b, nb, diag(S.K[q2].y, q.sc1 + rs, A.bA));
    }
    const int jo = j0 - 2;
    if (jo >= y0 && jo < row_end)
      store_pair<V>(A.out + (long long)jo * A.po, q.c0, max(gx + 2, 0), min(gx + 59, A.n), U);
  }
  // refill the slot of row t - 1, whose registers the black update above has consumed
  ps_issue<EDGE, V>(ring, A, t + PS_R - 1, T, y0, q, ci);
}

template <bool EDGE, bool V>
__device__ __forceinline__ void ps_run(unsigned char* ring, const PSArgs& A, int gx, int y0, int row_end) {
  const Lane q = lane_of(gx, A.n);
  const int ci = mirror_index(q.c0 >> 1, A.n >> 1);  // this lane's coarse column
  const int T = row_end - y0 + 4;
  PSState S;
#pragma unroll
  for (int k = 0; k < 4; ++k) S.U[k].a = S.U[k].b = make_float2(0.f, 0.f);
  S.Ee = make_float2(0.f, 0.f);
  for (int t = 0; t < PS_R - 1; ++t) ps_issue<EDGE, V>(ring, A, t, T, y0, q, ci);
#pragma unroll 1
  for (int t0 = 0; t0 < T; t0 += 2) {
    ps_stage<0, EDGE, V>(S, ring, A, t0 + 0, T, y0, row_end, gx, q, ci);
    ps_stage<1, EDGE, V>(S, ring, A, t0 + 1, T, y0, row_end, gx, q, ci);
    rotate2(S.U);
    rotate2(S.F);
    rotate2(S.K);
  }
  cp_wait<0>();
}

template <bool V>
__global__ void __launch_bounds__(32 * WPB) prolong_smooth_stream_kernel(PSArgs A, int strips, int seg_rows,
                                                                          const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * WPB + threadIdx.y;
  if (strip >= strips) return;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ring = smem + threadIdx.y * PS_R * PS_SLOT;
  A.out += blockIdx.z * bi.so;
  A.upre += blockIdx.z * bi.su;
  A.ec += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * PS_W - 2;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    ps_run<false, V>(ring, A, gx, y0, row_end);
  else
    ps_run<true, V>(ring, A, gx, y0, row_end);
}

bool aligned16(const void* p, long long pitch, long long stride) {
  return ((uintptr_t)p & 15) == 0 && !(pitch & 1) && !(stride & 1);
}

}  // namespace

// seg_rows: rows per warp (even, >= 2). u / upre and kh must have 16-byte aligned rows (even
// pitches, 16-byte aligned bases and instance strides); f and out may have any pitch.
cudaError_t launch_smooth_restrict_stream(void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                          int pk, int n, double bA, double bB, int seg_rows, const int* stop,
                                          cudaStream_t s, const Inst& bi) {
  if (seg_rows < 2 || (seg_rows & 1) || n < 4 || !aligned16(u, pu, bi.su) || !aligned16(kh, pk, 0))
    return cudaErrorInvalidValue;
  SRArgs A{(float2*)u, pu, (float2*)fc, pc, (const float2*)f, pf, (const float*)kh, pk, n, (float)bA, (float)bB};
  const int strips = (n + 1 + SR_W - 1) / SR_W, segs = (n + 1 + seg_rows - 1) / seg_rows;
  dim3 grid((strips + WPB - 1) / WPB, segs, bi.count);
  constexpr size_t sm = (size_t)WPB * SR_R * SR_SLOT;
  if (aligned16(f, pf, bi.sf))
    pdl_launch(smooth_restrict_stream_kernel<true>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  else
    pdl_launch(smooth_restrict_stream_kernel<false>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
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
  constexpr size_t sm = (size_t)WPB * PS_R * PS_SLOT;
  if (aligned16(f, pf, bi.sf) && aligned16(out, po, bi.so))
    pdl_launch(prolong_smooth_stream_kernel<true>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  else
    pdl_launch(prolong_smooth_stream_kernel<false>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  return cudaGetLastError();
}

}  // namespace hz
