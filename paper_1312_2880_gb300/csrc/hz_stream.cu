// Register-streaming forms of the two fused Gauss-Seidel passes (FP32 and FP64 forms).
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

template <class T>
struct L2c {  // a lane's two adjacent columns
  c2<T> a, b;
};

__device__ __forceinline__ int mirror_index(int i, int n) {
  i = i < 0 ? -i : i;
  i = i > n ? 2 * n - i : i;
  return i < 0 ? 0 : i;  // beyond one reflection: any node (such lanes never feed an output)
}
// Twice the boundary sides of row (or column) j, mirror images included (j in [-n, 2n]; n >= 1).
template <class T>
__device__ __forceinline__ T sides2(int j, int n) { return (j == 0 || j == n) ? (T)2 : (T)0; }

template <class T>
__device__ __forceinline__ c2<T> shfl_up2(c2<T> v) {
  return mk<T>(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}
template <class T>
__device__ __forceinline__ c2<T> shfl_down2(c2<T> v) {
  return mk<T>(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}
template <class T>
__device__ __forceinline__ c2<T> add2(c2<T> a, c2<T> b) { return xr::cadd<T>(a, b); }
template <class T>
__device__ __forceinline__ c2<T> scl2(c2<T> a, T s) { return xr::cscale<T>(a, s); }
template <class T>
__device__ __forceinline__ c2<T> diag(T k, T two_sides, T beta) { return xr::diag2<T>(k, two_sides, beta); }

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

// Asynchronous copy of one element of B = 4, 8 or 16 bytes.
template <int B>
__device__ __forceinline__ void cp_elem(unsigned dst, const void* src) {
  if constexpr (B == 16)
    cp16(dst, src);
  else if constexpr (B == 8)
    cp8(dst, src);
  else
    cp4(dst, src);
}
// A lane's pair of complex values from `row` into 2 sizeof(c2<T>) bytes at dst: in FP32 one 16-byte
// copy when the pair is contiguous and aligned (VEC, interior strips), else one copy per element
// (mirrored columns; in FP64 each element is 16 bytes anyway).
template <class T, bool EDGE, bool VEC>
__device__ __forceinline__ void copy_pair(unsigned dst, const c2<T>* row, int c0, int m0, int m1) {
  constexpr int E = sizeof(c2<T>);
  if (E == 8 && !EDGE && VEC) {
    cp16(dst, row + c0);
  } else {
    cp_elem<E>(dst, row + (EDGE ? m0 : c0));
    cp_elem<E>(dst + E, row + (EDGE ? m1 : c0 + 1));
  }
}
// The pair of k H values: in FP32 one 8-byte copy on interior strips (c0 is even and FP32 rows
// have even pitches), else one copy per value (FP64 rows of k H may have odd pitches).
template <class T, bool EDGE>
__device__ __forceinline__ void copy_kpair(unsigned dst, const T* row, int c0, int m0, int m1) {
  constexpr int E = sizeof(T);
  if (E == 4 && !EDGE) {
    cp8(dst, row + c0);
  } else if (!EDGE) {
    cp_elem<E>(dst, row + c0);
    cp_elem<E>(dst + E, row + c0 + 1);
  } else {
    cp_elem<E>(dst, row + m0);
    cp_elem<E>(dst + E, row + m1);
  }
}
template <class T>
__device__ __forceinline__ L2c<T> lds_pair(const unsigned char* p) {
  L2c<T> r;
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r.a = make_float2(v.x, v.y);
    r.b = make_float2(v.z, v.w);
  } else {
    r.a = reinterpret_cast<const double2*>(p)[0];
    r.b = reinterpret_cast<const double2*>(p)[1];
  }
  return r;
}

// Store a lane's pair where lo <= column <= hi (a lane stores both or, at the grid edge, one).
template <class T, bool VEC>
__device__ __forceinline__ void store_pair(c2<T>* __restrict__ row, int c0, int lo, int hi, const L2c<T>& U) {
  const bool s0 = c0 >= lo && c0 <= hi, s1 = c0 + 1 >= lo && c0 + 1 <= hi;
  if constexpr (sizeof(T) == 4) {
    if (VEC && s0 && s1) {
      *reinterpret_cast<float4*>(row + c0) = make_float4(U.a.x, U.a.y, U.b.x, U.b.y);
      return;
    }
  }
  if (s0) row[c0] = U.a;
  if (s1) row[c0 + 1] = U.b;
}

template <class T>
struct Lane {  // per-lane constants of a strip
  int c0, m0, m1;
  T sc0, sc1;  // twice the boundary sides of the two columns
};
template <class T>
__device__ __forceinline__ Lane<T> lane_of(int gx, int n) {
  Lane<T> q;
  q.c0 = gx + 2 * (int)threadIdx.x;
  q.m0 = mirror_index(q.c0, n);
  q.m1 = mirror_index(q.c0 + 1, n);
  q.sc0 = sides2<T>(q.c0, n);
  q.sc1 = sides2<T>(q.c0 + 1, n);
  return q;
}

// Bytes per lane in a ring slot: a pair of complex values (PE) and a pair of k H values (PK).
template <class T> __host__ __device__ constexpr int pair_bytes() { return 2 * (int)sizeof(c2<T>); }
template <class T> __host__ __device__ constexpr int kpair_bytes() { return 2 * (int)sizeof(T); }

// ------------------------------------------------------------------ smooth + residual + restrict
// Strip: columns gx .. gx + 63 with gx = 58 s - 4; the strip's outputs are columns gx + 4 ..
// gx + 61 (u) and coarse columns gx/2 + 2 .. gx/2 + 30. Segment: output rows y0 .. row_end - 1;
// loaded rows y0 - 3 .. row_end + 2, stage t handling loaded row t (global y0 - 3 + t):
//   red at row t, black at row t-1 (u of row t-1 final, stored), residual at row t-2 and its
//   full-weighting row sum (coarse row J completes at fine row 2J + 1).
constexpr int SR_W = 58;
constexpr int SR_R = 8;            // row slots per warp
// bytes per slot: f pairs (16 B per lane in FP32, 32 in FP64), then k pairs (8, 16)
template <class Real> __host__ __device__ constexpr int sr_slot() { return 32 * (pair_bytes<Real>() + kpair_bytes<Real>()); }

template <class Real>
struct SRArgs {
  c2<Real>* u;
  int pu;
  c2<Real>* fc;
  int pc;
  const c2<Real>* f;
  int pf;
  const Real* kh;
  int pk;
  int n;
  Real bA, bB;
};

template <class Real>
struct SRState {
  L2c<Real> F[4];
  c2<Real> K[4];
  L2c<Real> U[4];
  c2<Real> hS, hC;  // full-weighting row sums of rows 2J - 1 and 2J
};

template <class Real, bool EDGE, bool VF>
__device__ __forceinline__ void sr_issue(unsigned char* ring, const SRArgs<Real>& A, int t, int T, int y0, const Lane<Real>& q) {
  if (t < T) {
    const int mj = mirror_index(y0 - 3 + t, A.n);
    unsigned char* slot = ring + (t % SR_R) * sr_slot<Real>();
    copy_pair<Real, EDGE, VF>(smem_addr(slot + pair_bytes<Real>() * threadIdx.x), A.f + (long long)mj * A.pf, q.c0,
                              q.m0, q.m1);
    copy_kpair<Real, EDGE>(smem_addr(slot + 32 * pair_bytes<Real>() + kpair_bytes<Real>() * threadIdx.x),
                           A.kh + (long long)mj * A.pk, q.c0, q.m0, q.m1);
  }
  cp_commit();  // one group per row index, empty past the segment, so the wait count stays fixed
}

template <class Real, int Q, bool EDGE, bool VF>
__device__ __forceinline__ void sr_stage(SRState<Real>& S, unsigned char* ring, const SRArgs<Real>& A, int t, int T, int y0,
                                         int row_end, int gx, const Lane<Real>& q) {
  if (t >= T) return;
  cp_wait<SR_R - 2>();  // rows up to t have landed (t + R - 1 groups committed)
  {
    const unsigned char* slot = ring + (t % SR_R) * sr_slot<Real>();
    S.F[Q] = lds_pair<Real>(slot + pair_bytes<Real>() * threadIdx.x);
    S.K[Q] = *reinterpret_cast<const c2<Real>*>(slot + 32 * pair_bytes<Real>() + kpair_bytes<Real>() * threadIdx.x);
  }
  // global row y0 - 3 + t has the parity of t + 1: red is column 0 of the pair on odd t
  constexpr int er = (Q & 1) ? 0 : 1;
  const int j0 = y0 - 3 + t;
  {  // red at row t (zero guess)
    L2c<Real>& U = S.U[Q];
    const Real rs = sides2<Real>(j0, A.n);
    if (er == 0)
      U.a = xr::cdiv<Real>(S.F[Q].a, diag<Real>(S.K[Q].x, q.sc0 + rs, A.bA));
    else
      U.b = xr::cdiv<Real>(S.F[Q].b, diag<Real>(S.K[Q].y, q.sc1 + rs, A.bA));
  }
  if (t >= 1) {  // black at row t-1, column er
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3;
    const Real rs = sides2<Real>(j0 - 1, A.n);
    L2c<Real>& U = S.U[q1];
    if (er == 1) {
      const c2<Real> nb = xr::nb4<Real>(U.a, shfl_down2<Real>(U.a), S.U[q2].b, S.U[Q].b);
      U.b = xr::gs<Real>(S.F[q1].b, nb, diag<Real>(S.K[q1].y, q.sc1 + rs, A.bA));
    } else {
      const c2<Real> nb = xr::nb4<Real>(shfl_up2<Real>(U.b), U.b, S.U[q2].a, S.U[Q].a);
      U.a = xr::gs<Real>(S.F[q1].a, nb, diag<Real>(S.K[q1].x, q.sc0 + rs, A.bA));
    }
    const int jo = j0 - 1;
    if (jo >= y0 && jo < row_end) store_pair<Real, true>(A.u + (long long)jo * A.pu, q.c0, gx + 4, min(gx + 61, A.n), U);
  }
  if (t >= 2) {  // residual f - B u at row t-2 and its full-weighting row sum
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3, q3 = (Q + 1) & 3;
    const Real rs = sides2<Real>(j0 - 2, A.n);
    const L2c<Real>& U = S.U[q2];
    L2c<Real> R;
    R.a = xr::resid<Real>(S.F[q2].a, U.a, xr::nb4<Real>(shfl_up2<Real>(U.b), U.b, S.U[q3].a, S.U[q1].a),
                           diag<Real>(S.K[q2].x, q.sc0 + rs, A.bB));
    R.b = xr::resid<Real>(S.F[q2].b, U.b, xr::nb4<Real>(U.a, shfl_down2<Real>(U.a), S.U[q3].b, S.U[q1].b),
                           diag<Real>(S.K[q2].y, q.sc1 + rs, A.bB));
    // the row sum (w + e) + 2 c at this lane's coarse column (2I = c0), then across rows; row
    // j0 - 2 is even (2J) on odd t, odd (2J + 1) on even t
    const c2<Real> h = xr::fw3<Real>(shfl_up2<Real>(R.b), R.a, R.b);
    if (Q & 1) {
      S.hC = h;
    } else {
      const int j2 = j0 - 3;  // = 2J
      if (j2 >= y0 && j2 < row_end) {
        const int L = threadIdx.x, I = (gx >> 1) + L;
        if (L >= 2 && L <= 30 && I <= (A.n >> 1))
          A.fc[(long long)(j2 >> 1) * A.pc + I] = scl2<Real>(xr::fw3<Real>(S.hS, S.hC, h), (Real)0.25);
      }
      S.hS = h;
    }
  }
  // refill the slot of row t - 1, whose registers the black update above has consumed
  sr_issue<Real, EDGE, VF>(ring, A, t + SR_R - 1, T, y0, q);
}

template <class Real, bool EDGE, bool VF>
__device__ __forceinline__ void sr_run(unsigned char* ring, const SRArgs<Real>& A, int gx, int y0, int row_end) {
  const Lane<Real> q = lane_of<Real>(gx, A.n);
  const int T = row_end - y0 + 6;
  SRState<Real> S;
#pragma unroll
  for (int k = 0; k < 4; ++k) S.U[k].a = S.U[k].b = mk<Real>(0, 0);
  S.hS = S.hC = mk<Real>(0, 0);
  for (int t = 0; t < SR_R - 1; ++t) sr_issue<Real, EDGE, VF>(ring, A, t, T, y0, q);
  // four stages of code per iteration, one per slot of the four-row windows (row t in slot
  // t mod 4), so no register moves rotate the windows between iterations
#pragma unroll 1
  for (int t0 = 0; t0 < T; t0 += 4) {
    sr_stage<Real, 0, EDGE, VF>(S, ring, A, t0 + 0, T, y0, row_end, gx, q);
    sr_stage<Real, 1, EDGE, VF>(S, ring, A, t0 + 1, T, y0, row_end, gx, q);
    sr_stage<Real, 2, EDGE, VF>(S, ring, A, t0 + 2, T, y0, row_end, gx, q);
    sr_stage<Real, 3, EDGE, VF>(S, ring, A, t0 + 3, T, y0, row_end, gx, q);
  }
  cp_wait<0>();
}

template <class Real, bool VF>
__global__ void __launch_bounds__(32 * WPB) smooth_restrict_stream_kernel(SRArgs<Real> A, int strips, int seg_rows,
                                                                           const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * WPB + threadIdx.y;
  if (strip >= strips) return;  // whole warp
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ring = smem + threadIdx.y * SR_R * sr_slot<Real>();
  A.u += blockIdx.z * bi.su;
  A.fc += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * SR_W - 4;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    sr_run<Real, false, VF>(ring, A, gx, y0, row_end);
  else
    sr_run<Real, true, VF>(ring, A, gx, y0, row_end);
}

// ------------------------------------------------------------------ prolong + post-smooth
// Strip: columns gx .. gx + 63 with gx = 58 s - 2; outputs gx + 2 .. gx + 59 (v = u_pre + P e_c
// is valid on gx .. gx + 62: the odd column of the last lane would need the next lane's coarse
// value; black nodes on gx + 1 .. gx + 61; red on gx + 2 .. gx + 60). Loaded rows y0 - 2 ..
// row_end + 1, plus the coarse row under row_end + 2 when row_end + 1 is odd; stage t: v at row t,
// black at row t-1 (from v), red at row t-2 (from the updated black nodes), row t-2 stored.
constexpr int PS_W = 58;
constexpr int PS_R = 8;            // row slots per warp
// bytes per slot: f pairs (16 B per lane in FP32, 32 in FP64), u_pre pairs (16, 32), k pairs (8,
// 16), coarse e (8, 16)
template <class Real> __host__ __device__ constexpr int ps_upre_off() { return 32 * pair_bytes<Real>(); }
template <class Real> __host__ __device__ constexpr int ps_k_off() { return 64 * pair_bytes<Real>(); }
template <class Real> __host__ __device__ constexpr int ps_e_off() { return ps_k_off<Real>() + 32 * kpair_bytes<Real>(); }
template <class Real> __host__ __device__ constexpr int ps_slot() { return ps_e_off<Real>() + 32 * (int)sizeof(c2<Real>); }

template <class Real>
struct PSArgs {
  c2<Real>* out;
  int po;
  const c2<Real>* upre;
  int pu;
  const c2<Real>* ec;
  int pc;
  const c2<Real>* f;
  int pf;
  const Real* kh;
  int pk;
  int n;
  Real bA;
};

template <class Real>
struct PSState {
  L2c<Real> F[4];
  c2<Real> K[4];
  L2c<Real> U[4];
  c2<Real> Ee;  // coarse e under the last even row
};

// Copies of loaded row t (< T) and, on even rows, of the coarse row under it (also for t == T,
// which the odd row T - 1 interpolates from).
template <class Real, bool EDGE, bool V>
__device__ __forceinline__ void ps_issue(unsigned char* ring, const PSArgs<Real>& A, int t, int T, int y0, const Lane<Real>& q,
                                         int ci) {
  if (t <= T) {
    const int j = y0 - 2 + t;
    unsigned char* slot = ring + (t % PS_R) * ps_slot<Real>();
    if (t < T) {
      const int mj = mirror_index(j, A.n);
      copy_pair<Real, EDGE, V>(smem_addr(slot + pair_bytes<Real>() * threadIdx.x), A.f + (long long)mj * A.pf, q.c0,
                               q.m0, q.m1);
      copy_pair<Real, EDGE, true>(smem_addr(slot + ps_upre_off<Real>() + pair_bytes<Real>() * threadIdx.x),
                                  A.upre + (long long)mj * A.pu, q.c0, q.m0, q.m1);
      copy_kpair<Real, EDGE>(smem_addr(slot + ps_k_off<Real>() + kpair_bytes<Real>() * threadIdx.x),
                             A.kh + (long long)mj * A.pk, q.c0, q.m0, q.m1);
    }
    if (!(j & 1))
      cp_elem<sizeof(c2<Real>)>(smem_addr(slot + ps_e_off<Real>() + (int)sizeof(c2<Real>) * threadIdx.x),
                                A.ec + (long long)mirror_index(j >> 1, A.n >> 1) * A.pc + ci);
  }
  cp_commit();
}

template <class Real, int Q, bool EDGE, bool V>
__device__ __forceinline__ void ps_stage(PSState<Real>& S, unsigned char* ring, const PSArgs<Real>& A, int t, int T, int y0,
                                         int row_end, int gx, const Lane<Real>& q, int ci) {
  if (t >= T) return;
  cp_wait<PS_R - 3>();  // rows up to t + 1 have landed (t + R - 1 groups committed)
  const unsigned char* slot = ring + (t % PS_R) * ps_slot<Real>();
  S.F[Q] = lds_pair<Real>(slot + pair_bytes<Real>() * threadIdx.x);
  S.K[Q] = *reinterpret_cast<const c2<Real>*>(slot + ps_k_off<Real>() + kpair_bytes<Real>() * threadIdx.x);
  // global row y0 - 2 + t has the parity of t: red is column 0 of the pair on even t
  constexpr int er = (Q & 1) ? 1 : 0;
  const int j0 = y0 - 2 + t;
  {  // v = u_pre + P e at row t
    const L2c<Real> up = lds_pair<Real>(slot + ps_upre_off<Real>() + pair_bytes<Real>() * threadIdx.x);
    L2c<Real>& U = S.U[Q];
    if (Q & 1) {
      const unsigned char* next = ring + ((t + 1) % PS_R) * ps_slot<Real>();
      const c2<Real> ev =
          add2<Real>(S.Ee, *reinterpret_cast<const c2<Real>*>(next + ps_e_off<Real>() + (int)sizeof(c2<Real>) * threadIdx.x));
      U.a = add2<Real>(up.a, scl2<Real>(ev, (Real)0.5));
      U.b = add2<Real>(up.b, scl2<Real>(add2<Real>(ev, shfl_down2<Real>(ev)), (Real)0.25));
    } else {
      S.Ee = *reinterpret_cast<const c2<Real>*>(slot + ps_e_off<Real>() + (int)sizeof(c2<Real>) * threadIdx.x);
      U.a = add2<Real>(up.a, S.Ee);
      U.b = add2<Real>(up.b, scl2<Real>(add2<Real>(S.Ee, shfl_down2<Real>(S.Ee)), (Real)0.5));
    }
  }
  if (t >= 1) {  // black at row t-1, column er (its vertical neighbours are red v nodes)
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3;
    const Real rs = sides2<Real>(j0 - 1, A.n);
    L2c<Real>& U = S.U[q1];
    if (er == 1) {
      const c2<Real> nb = xr::nb4<Real>(U.a, shfl_down2<Real>(U.a), S.U[q2].b, S.U[Q].b);
      U.b = xr::gs<Real>(S.F[q1].b, nb, diag<Real>(S.K[q1].y, q.sc1 + rs, A.bA));
    } else {
      const c2<Real> nb = xr::nb4<Real>(shfl_up2<Real>(U.b), U.b, S.U[q2].a, S.U[Q].a);
      U.a = xr::gs<Real>(S.F[q1].a, nb, diag<Real>(S.K[q1].x, q.sc0 + rs, A.bA));
    }
  }
  if (t >= 2) {  // red at row t-2, column er (its neighbours are updated black nodes)
    constexpr int q1 = (Q + 3) & 3, q2 = (Q + 2) & 3, q3 = (Q + 1) & 3;
    const Real rs = sides2<Real>(j0 - 2, A.n);
    L2c<Real>& U = S.U[q2];
    if (er == 0) {
      const c2<Real> nb = xr::nb4<Real>(shfl_up2<Real>(U.b), U.b, S.U[q3].a, S.U[q1].a);
      U.a = xr::gs<Real>(S.F[q2].a, nb, diag<Real>(S.K[q2].x, q.sc0 + rs, A.bA));
    } else {
      const c2<Real> nb = xr::nb4<Real>(U.a, shfl_down2<Real>(U.a), S.U[q3].b, S.U[q1].b);
      U.b = xr::gs<Real>(S.F[q2].b, nb, diag<Real>(S.K[q2].y, q.sc1 + rs, A.bA));
    }
    const int jo = j0 - 2;
    if (jo >= y0 && jo < row_end)
      store_pair<Real, V>(A.out + (long long)jo * A.po, q.c0, max(gx + 2, 0), min(gx + 59, A.n), U);
  }
  // refill the slot of row t - 1, whose registers the black update above has consumed
  ps_issue<Real, EDGE, V>(ring, A, t + PS_R - 1, T, y0, q, ci);
}

template <class Real, bool EDGE, bool V>
__device__ __forceinline__ void ps_run(unsigned char* ring, const PSArgs<Real>& A, int gx, int y0, int row_end) {
  const Lane<Real> q = lane_of<Real>(gx, A.n);
  const int ci = mirror_index(q.c0 >> 1, A.n >> 1);  // this lane's coarse column
  const int T = row_end - y0 + 4;
  PSState<Real> S;
#pragma unroll
  for (int k = 0; k < 4; ++k) S.U[k].a = S.U[k].b = mk<Real>(0, 0);
  S.Ee = mk<Real>(0, 0);
  for (int t = 0; t < PS_R - 1; ++t) ps_issue<Real, EDGE, V>(ring, A, t, T, y0, q, ci);
#pragma unroll 1
  for (int t0 = 0; t0 < T; t0 += 4) {  // as in sr_run: row t in window slot t mod 4
    ps_stage<Real, 0, EDGE, V>(S, ring, A, t0 + 0, T, y0, row_end, gx, q, ci);
    ps_stage<Real, 1, EDGE, V>(S, ring, A, t0 + 1, T, y0, row_end, gx, q, ci);
    ps_stage<Real, 2, EDGE, V>(S, ring, A, t0 + 2, T, y0, row_end, gx, q, ci);
    ps_stage<Real, 3, EDGE, V>(S, ring, A, t0 + 3, T, y0, row_end, gx, q, ci);
  }
  cp_wait<0>();
}

template <class Real, bool V>
__global__ void __launch_bounds__(32 * WPB) prolong_smooth_stream_kernel(PSArgs<Real> A, int strips, int seg_rows,
                                                                          const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  const int strip = blockIdx.x * WPB + threadIdx.y;
  if (strip >= strips) return;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ring = smem + threadIdx.y * PS_R * ps_slot<Real>();
  A.out += blockIdx.z * bi.so;
  A.upre += blockIdx.z * bi.su;
  A.ec += blockIdx.z * bi.sc;
  A.f += blockIdx.z * bi.sf;
  const int gx = strip * PS_W - 2;
  const int y0 = blockIdx.y * seg_rows;
  const int row_end = min(y0 + seg_rows, A.n + 1);
  if (gx >= 0 && gx + 63 <= A.n)
    ps_run<Real, false, V>(ring, A, gx, y0, row_end);
  else
    ps_run<Real, true, V>(ring, A, gx, y0, row_end);
}

bool aligned16(const void* p, long long pitch, long long stride) {
  return ((uintptr_t)p & 15) == 0 && !(pitch & 1) && !(stride & 1);
}

// Dynamic shared memory above the default 48 KB (the FP64 rings), set once per kernel.
template <class K>
cudaError_t allow_smem(K kernel, size_t bytes, bool& done) {
  if (done || bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (!e) done = true;
  return e;
}

template <class Real>
cudaError_t sr_stream(void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh, int pk, int n,
                      double bA, double bB, int seg_rows, const int* stop, cudaStream_t s, const Inst& bi) {
  SRArgs<Real> A{(c2<Real>*)u, pu, (c2<Real>*)fc, pc, (const c2<Real>*)f, pf, (const Real*)kh, pk, n, (Real)bA, (Real)bB};
  const int strips = (n + 1 + SR_W - 1) / SR_W, segs = (n + 1 + seg_rows - 1) / seg_rows;
  dim3 grid((strips + WPB - 1) / WPB, segs, bi.count);
  constexpr size_t sm = (size_t)WPB * SR_R * sr_slot<Real>();
  static bool ready[2] = {false, false};
  cudaError_t e;
  if (aligned16(f, pf, bi.sf)) {
    if ((e = allow_smem(smooth_restrict_stream_kernel<Real, true>, sm, ready[1]))) return e;
    pdl_launch(smooth_restrict_stream_kernel<Real, true>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  } else {
    if ((e = allow_smem(smooth_restrict_stream_kernel<Real, false>, sm, ready[0]))) return e;
    pdl_launch(smooth_restrict_stream_kernel<Real, false>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  }
  return cudaGetLastError();
}

template <class Real>
cudaError_t ps_stream(void* out, int po, const void* upre, int pu, const void* ec, int pc, const void* f, int pf,
                      const void* kh, int pk, int n, double bA, int seg_rows, const int* stop, cudaStream_t s,
                      const Inst& bi) {
  PSArgs<Real> A{(c2<Real>*)out, po, (const c2<Real>*)upre, pu, (const c2<Real>*)ec, pc, (const c2<Real>*)f, pf,
                 (const Real*)kh, pk, n, (Real)bA};
  const int strips = (n + 1 + PS_W - 1) / PS_W, segs = (n + 1 + seg_rows - 1) / seg_rows;
  dim3 grid((strips + WPB - 1) / WPB, segs, bi.count);
  constexpr size_t sm = (size_t)WPB * PS_R * ps_slot<Real>();
  static bool ready[2] = {false, false};
  cudaError_t e;
  if (aligned16(f, pf, bi.sf) && aligned16(out, po, bi.so)) {
    if ((e = allow_smem(prolong_smooth_stream_kernel<Real, true>, sm, ready[1]))) return e;
    pdl_launch(prolong_smooth_stream_kernel<Real, true>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  } else {
    if ((e = allow_smem(prolong_smooth_stream_kernel<Real, false>, sm, ready[0]))) return e;
    pdl_launch(prolong_smooth_stream_kernel<Real, false>, grid, dim3(32, WPB), sm, s, A, strips, seg_rows, stop, bi);
  }
  return cudaGetLastError();
}

}  // namespace

// seg_rows: rows per warp (even, >= 2). FP32: u / upre and kh must have 16-byte aligned rows
// (even pitches, 16-byte aligned bases and instance strides); f and out may have any pitch. FP64:
// any pitches (every complex element is 16-byte aligned).
cudaError_t launch_smooth_restrict_stream(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf,
                                          const void* kh, int pk, int n, double bA, double bB, int seg_rows,
                                          const int* stop, cudaStream_t s, const Inst& bi) {
  if (seg_rows < 2 || (seg_rows & 1) || n < 4 || (fp32 && (!aligned16(u, pu, bi.su) || !aligned16(kh, pk, 0))))
    return cudaErrorInvalidValue;
  return fp32 ? sr_stream<float>(u, pu, fc, pc, f, pf, kh, pk, n, bA, bB, seg_rows, stop, s, bi)
              : sr_stream<double>(u, pu, fc, pc, f, pf, kh, pk, n, bA, bB, seg_rows, stop, s, bi);
}

cudaError_t launch_prolong_smooth_stream(bool fp32, void* out, int po, const void* upre, int pu, const void* ec, int pc,
                                         const void* f, int pf, const void* kh, int pk, int n, double bA, int seg_rows,
                                         const int* stop, cudaStream_t s, const Inst& bi) {
  if (seg_rows < 2 || (seg_rows & 1) || n < 4 ||
      (fp32 && (!aligned16(upre, pu, bi.su) || !aligned16(kh, pk, 0))))
    return cudaErrorInvalidValue;
  return fp32 ? ps_stream<float>(out, po, upre, pu, ec, pc, f, pf, kh, pk, n, bA, seg_rows, stop, s, bi)
              : ps_stream<double>(out, po, upre, pu, ec, pc, f, pf, kh, pk, n, bA, seg_rows, stop, s, bi);
}

}  // namespace hz
