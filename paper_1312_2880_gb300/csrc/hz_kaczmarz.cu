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
// kacz_sweep_tile: one or two full sweeps (all five colours each) per launch over tiles with a halo
//   that holds the dependency cone of the sweeps (6 columns each side, 6 and 10 rows per sweep), so
//   the tile interior holds exactly the sequential sweeps' values; each phase acts only on the
//   part of the region that can still reach the tile. Out of place.
// kacz_cluster_*: the kacz_level_* operations with the level split into row bands over a
//   thread-block cluster of up to 16 blocks (distributed shared memory, one cluster barrier per
//   colour), for levels too large for one block or, in FP64, too slow on one SM's FP64 pipe.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "hz_common.cuh"
#include "hz_internal.h"
#include "hz_level.cuh"

namespace hz {

namespace {

constexpr int LB = 1024;  // threads of the whole-level kernel
// Tiles of the tiled form: KT x KT outputs per block after S sweeps per launch. The halo is the
// dependency cone of S five-colour sweeps (found by propagating dependencies through the colour
// phases on an unbounded grid, every residue of the colour pattern): after one sweep in the order
// 0..4 an output depends on starting values at most 6 columns to either side, 6 rows below and 10
// rows above; in the order 4..0 the rows swap (10 below, 6 above); S sweeps add up the extents.
template <int KT_, int S_, int TB_>
struct TileGeo {
  static constexpr int KT = KT_, S = S_, TBK = TB_;
  static constexpr int HX = 6 * S_;             // halo columns on each side
  static constexpr int HN = 6 * S_, HF = 10 * S_;  // halo rows on the near and the far side
  static constexpr int RX = KT_ + 2 * HX, RY = KT_ + HN + HF, REG = RX * RY;
};
using TileOne = TileGeo<32, 1, 256>;   // one sweep per launch: 44 x 48 regions
using TileTwo = TileGeo<64, 2, 1024>;  // two sweeps per launch: 88 x 96 regions (FP32, n_l >= 1024)
using TileTwoS = TileGeo<32, 2, 512>;  // two sweeps per launch: 56 x 64 regions (FP32, n_l = 256 .. 1023)
template <class T, class G>
constexpr size_t tile_smem() { return (size_t)G::REG * (2 * sizeof(c2<T>) + sizeof(T)); }

// Actions of phase ph (of P = 5S; R = P - 1 - ph phases follow it) that can still reach the
// tile's outputs. Propagating dependencies back from the outputs through the colour phases on an
// unbounded grid (every residue of the colour pattern gives the same bounds) leaves, in tile
// coordinates (output origin 0), the phase's colour in columns -1-R .. KT+R and rows -1-R .. KT+2R
// (order 0..4) or -1-2R .. KT+R (order 4..0). An action outside that rectangle changes only values
// no output depends on, so leaving it out keeps the outputs' bits, and it cuts the actions of a
// two-sweep launch on 64-node tiles by a third against sweeping the whole region every phase.
// Slot q of a phase is the (q mod per)-th node of the colour from column xlo in row ylo + q / per.
template <class G, bool POST>
struct PhaseRect {
  static constexpr int P = 5 * G::S;
  static constexpr int below = POST ? G::HF : G::HN;  // region rows below the tile
  __host__ __device__ static constexpr int R(int ph) { return P - 1 - ph; }
  __host__ __device__ static constexpr int xlo(int ph) { return G::HX - 1 - R(ph); }
  __host__ __device__ static constexpr int xhi(int ph) { return G::HX + G::KT + R(ph); }
  __host__ __device__ static constexpr int ylo(int ph) { return below - 1 - (POST ? 2 : 1) * R(ph); }
  __host__ __device__ static constexpr int yhi(int ph) { return below + G::KT + (POST ? 1 : 2) * R(ph); }
  __host__ __device__ static constexpr int per(int ph) { return (xhi(ph) - xlo(ph)) / 5 + 1; }
  __host__ __device__ static constexpr int slots(int ph) { return (yhi(ph) - ylo(ph) + 1) * per(ph); }
  // every rectangle's supports inside the region, at most two slots per thread
  __host__ __device__ static constexpr bool fits() {
    for (int ph = 0; ph < P; ++ph)
      if (xlo(ph) < 1 || xhi(ph) > G::RX - 2 || ylo(ph) < 1 || yhi(ph) > G::RY - 2 || slots(ph) > 2 * G::TBK)
        return false;
    return true;
  }
};

// One slot's row action: shared offsets of the node and its W, E, S, N support (a mirror neighbour
// at the boundary appears twice), the values read, and the row's right-hand side and constants.
template <class T>
struct TileAct {
  int op, ow, oe, os, on, i, j;
  bool ok, mx, my;
  c2<T> up, uw, ue, us, un, f;
};

__device__ __forceinline__ int mod5(int x) { return ((x % 5) + 5) % 5; }

// Phase PH of a tile: each thread takes up to two slots, reads both supports before updating
// either (same-colour supports are disjoint), then writes both back. The row constants come from
// k H as in the whole-level forms (lvl::row_consts; strictly inside the square, no boundary term)
// and the arithmetic is lvl::act_update, so a tiled sweep gives the same bits as the whole-level
// and cluster forms.
template <class T, class G, bool POST, bool INNER, int PH>
__device__ __forceinline__ void tile_phase(c2<T>* su, const c2<T>* sf, const T* sk, const unsigned char* c0row,
                                           int gx, int gy, int n, T beta) {
  using PR = PhaseRect<G, POST>;
  constexpr int colour = POST ? 4 - PH % 5 : PH % 5;
  constexpr int xlo = PR::xlo(PH), xhi = PR::xhi(PH), ylo = PR::ylo(PH), per = PR::per(PH), slots = PR::slots(PH);
  constexpr int K = ((colour - xlo) % 5 + 5) % 5;
  constexpr int NS = slots > G::TBK ? 2 : 1;
  constexpr int W = G::RX;
  TileAct<T> a[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int q = (int)threadIdx.x + s * G::TBK;
    const int rr = q / per, m = q - rr * per, r = ylo + rr;
    int t = (q < slots ? (int)c0row[r] : 0) + K;  // column residue of the colour in row r, from xlo
    t -= t >= 5 ? 5 : 0;
    const int c = xlo + t + 5 * m, p = r * W + c;
    TileAct<T>& A = a[s];
    A.ok = q < slots && c <= xhi;
    A.op = p;
    if constexpr (INNER) {
      A.mx = A.my = false;
      A.ow = p - 1;
      A.oe = p + 1;
      A.os = p - W;
      A.on = p + W;
    } else {
      A.i = gx + c;
      A.j = gy + r;
      A.ok = A.ok && (unsigned)A.i <= (unsigned)n && (unsigned)A.j <= (unsigned)n;
      A.mx = A.i == 0 || A.i == n;
      A.my = A.j == 0 || A.j == n;
      A.ow = p + (A.i > 0 ? -1 : 1);
      A.oe = p + (A.i < n ? 1 : -1);
      A.os = p + (A.j > 0 ? -W : W);
      A.on = p + (A.j < n ? W : -W);
    }
  }
  T kh[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    TileAct<T>& A = a[s];
    if (A.ok) {
      A.up = su[A.op];
      A.uw = su[A.ow];
      A.ue = su[A.oe];
      A.us = su[A.os];
      A.un = su[A.on];
      A.f = sf[A.op];
      kh[s] = sk[A.op];
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    TileAct<T>& A = a[s];
    if (A.ok) {
      c2<T> d;
      T inv;
      if constexpr (INNER) {
        d = xr::diag<T>(kh[s], 0, beta);
        inv = xr::rcp(xr::add(xr::cabs2<T>(d), (T)4));
      } else {
        lvl::row_consts<T>(kh[s], A.i, A.j, n, beta, &d, &inv);
      }
      lvl::act_update<T>(A.up, A.uw, A.ue, A.us, A.un, A.f, d, inv, A.mx, A.my);
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const TileAct<T>& A = a[s];
    if (A.ok) {
      su[A.op] = A.up;
      su[A.ow] = A.uw;
      if (!A.mx) su[A.oe] = A.ue;
      su[A.os] = A.us;
      if (!A.my) su[A.on] = A.un;
    }
  }
}

// All phases of a launch in order, a barrier after each.
template <class T, class G, bool POST, bool INNER, int... PH>
__device__ __forceinline__ void tile_phases(c2<T>* su, const c2<T>* sf, const T* sk, const unsigned char* c0row,
                                            int gx, int gy, int n, T beta, std::integer_sequence<int, PH...>) {
  ((tile_phase<T, G, POST, INNER, PH>(su, sf, sk, c0row, gx, gy, n, beta), __syncthreads()), ...);
}

// ------------------------------------------------------------------ whole level in one block
// Shared layout of the whole-level kernels: u, f~, d (complex) and 1/|a|^2 (real) per node, each
// array colour-blocked (lvl::Blocked, N = lvl::blocked_cells(n) cells).
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

// Global <-> shared copies visit the level in row-major order (coalesced on the global side) and
// go through cp.async, one wait for all of them: a load per node at a time would put one memory
// latency per node a thread holds on the launch's critical path. k H (fixed per problem) and the
// zero guess are issued before the wait for the preceding kernel. The row constants then replace
// k H in place.
template <class T>
__device__ __forceinline__ void level_kh_async(const LevelSmem<T>& S, const T* kh, int pk, int n) {
  lvl::for_nodes_blocked(n, [&](int, int i, int j, int p) {
    lvl::cp_async<sizeof(T)>(&S.sinv[p], kh + (long long)j * pk + i);
  });
}
template <class T>
__device__ __forceinline__ void level_row_consts(const LevelSmem<T>& S, int n, T bA) {
  lvl::for_blocked(n, [&](int i, int j, int p) { lvl::row_consts<T>(S.sinv[p], i, j, n, bA, &S.sd[p], &S.sinv[p]); });
}

template <class T>
__global__ void __launch_bounds__(LB) kacz_level_pre_kernel(c2<T>* __restrict__ u, int pu, c2<T>* __restrict__ fc,
                                                             int pc, const c2<T>* __restrict__ f, int pf,
                                                             const T* __restrict__ kh, int pk, int n, T bA, T bB,
                                                             int nu, const int* __restrict__ stop, Inst bi) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Np = lvl::blocked_cells(n);
  LevelSmem<T> S(smem, Np);
  for (int q = threadIdx.x; q < Np; q += LB) S.su[q] = mk<T>(0, 0);
  level_kh_async<T>(S, kh, pk, n);
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) {
    lvl::cp_async_wait_all();
    return;
  }
  u += blockIdx.z * bi.su;
  fc += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  lvl::for_nodes_blocked(n, [&](int, int i, int j, int p) {
    lvl::cp_async<sizeof(c2<T>)>(&S.sf[p], f + (long long)j * pf + i);
  });
  lvl::cp_async_wait_all();
  __syncthreads();
  level_row_consts<T>(S, n, bA);
  __syncthreads();
  lvl::kacz_sweeps<T>(S.su, S.sf, S.sd, S.sinv, n, nu, false);
  lvl::for_nodes_blocked(n, [&](int, int i, int j, int p) { u[(long long)j * pu + i] = S.su[p]; });
  lvl::residual_blocked<T>(S.sd, S.su, S.sf, kh, pk, n, bB);  // the residual (natural) replaces the diagonals
  __syncthreads();
  lvl::restrict_fw<T>(fc, lvl::Natural{pc}, S.sd, n);
}

template <class T>
__global__ void __launch_bounds__(LB) kacz_level_post_kernel(c2<T>* __restrict__ u, int pu,
                                                              const c2<T>* __restrict__ ec, int pc,
                                                              const c2<T>* __restrict__ f, int pf,
                                                              const T* __restrict__ kh, int pk, int n, T bA, int nu,
                                                              const int* __restrict__ stop, Inst bi) {
  extern __shared__ __align__(16) unsigned char smem[];
  LevelSmem<T> S(smem, lvl::blocked_cells(n));
  level_kh_async<T>(S, kh, pk, n);
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) {
    lvl::cp_async_wait_all();
    return;
  }
  u += blockIdx.z * bi.su;
  ec += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  // u and f into their cells, the coarse correction row-major (pitch wc) into the diagonals' cells
  const int wc = n / 2 + 1;
  lvl::for_nodes_blocked(n, [&](int, int i, int j, int p) {
    lvl::cp_async<sizeof(c2<T>)>(&S.su[p], u + (long long)j * pu + i);
    lvl::cp_async<sizeof(c2<T>)>(&S.sf[p], f + (long long)j * pf + i);
  });
  lvl::for_nodes(wc, wc * wc, [&](int q, int I, int J) {
    lvl::cp_async<sizeof(c2<T>)>(&S.sd[q], ec + (long long)J * pc + I);
  });
  lvl::cp_async_wait_all();
  __syncthreads();
  lvl::for_blocked(n, [&](int i, int j, int p) {
    const c2<T>* e0 = S.sd + (j >> 1) * wc;
    S.su[p] = xr::cadd<T>(S.su[p], xr::bilinear<T>(e0, e0 + wc, i >> 1, i & 1, j & 1));
  });
  __syncthreads();
  level_row_consts<T>(S, n, bA);
  __syncthreads();
  lvl::kacz_sweeps<T>(S.su, S.sf, S.sd, S.sinv, n, nu, true);
  lvl::for_nodes_blocked(n, [&](int, int i, int j, int p) { u[(long long)j * pu + i] = S.su[p]; });
}

template <class T, class F2, class G, bool POST>
__device__ __forceinline__ void tile_sweeps(c2<T>* __restrict__ uout, int po, const c2<T>* __restrict__ uin, int pu,
                                            const F2* __restrict__ f, int pf, const T* __restrict__ kh, int pk, int n,
                                            T bA, const int* __restrict__ stop, Inst bi) {
  using PR = PhaseRect<G, POST>;
  static_assert(PR::fits(), "phase rectangles must keep their supports inside the tile region");
  constexpr int TBK = G::TBK, RX = G::RX, RY = G::RY, REG = G::REG, KT = G::KT;
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  uout += blockIdx.z * bi.su;
  if (uin) uin += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T>* su = reinterpret_cast<c2<T>*>(smem);
  c2<T>* sf = su + REG;
  T* sk = reinterpret_cast<T*>(sf + REG);
  __shared__ unsigned char c0row[RY];  // column residue of colour 0 in each region row
  const int x0 = blockIdx.x * KT, y0 = blockIdx.y * KT;
  // sweeps in the order 0..4 (pre) need the near halo below the tile, 4..0 (post) above it
  constexpr int below = PR::below;
  const int gx = x0 - G::HX, gy = y0 - below;
  // the tile region's u, f~ and k H in flight at once (cp.async, one wait): a plain load per node
  // would put one L2 latency per node a thread copies on the launch's critical path. A warp
  // takes whole region rows, a lane every 32nd column: no division per node.
  constexpr bool async_f = sizeof(F2) == sizeof(c2<T>);  // f~ in the level's own precision
  constexpr int NW = TBK / 32;
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  for (int r = warp; r < RY; r += NW) {
    const int j = gy + r;
    if ((unsigned)j > (unsigned)n) continue;
    const long long ju = (long long)j * pu, jf = (long long)j * pf, jk = (long long)j * pk;
    for (int c = lane; c < RX; c += 32) {
      const int i = gx + c, q = r * RX + c;
      if ((unsigned)i > (unsigned)n) continue;
      if (uin)
        lvl::cp_async<sizeof(c2<T>)>(su + q, uin + ju + i);
      else
        su[q] = mk<T>(0, 0);
      if constexpr (async_f)
        lvl::cp_async<sizeof(c2<T>)>(sf + q, f + jf + i);
      else
        sf[q] = ldc<T>(f, jf + i);
      lvl::cp_async<sizeof(T)>(sk + q, kh + jk + i);
    }
  }
  for (int r = threadIdx.x; r < RY; r += TBK) c0row[r] = (unsigned char)mod5(-2 * (gy + r) - gx);
  lvl::cp_async_wait_all();
  __syncthreads();
  // every action strictly inside the square: no mirrors, no boundary terms (phase 0's rectangle
  // holds every later one)
  const bool inner = gx + PR::xlo(0) >= 1 && gx + PR::xhi(0) <= n - 1 && gy + PR::ylo(0) >= 1 &&
                     gy + PR::yhi(0) <= n - 1;
  if (inner)
    tile_phases<T, G, POST, true>(su, sf, sk, c0row, gx, gy, n, bA, std::make_integer_sequence<int, PR::P>{});
  else
    tile_phases<T, G, POST, false>(su, sf, sk, c0row, gx, gy, n, bA, std::make_integer_sequence<int, PR::P>{});
  // the tile's own KT x KT nodes (those inside the square) back to global memory, rows by warp
  for (int r = below + warp; r < below + KT; r += NW) {
    const int j = gy + r;
    if (j > n) break;
    c2<T>* orow = uout + (long long)j * po;
    for (int c = G::HX + lane; c < G::HX + KT; c += 32) {
      const int i = gx + c;
      if (i > n) break;
      orow[i] = su[r * RX + c];
    }
  }
}

// FP32 tiles are held to 56 registers a thread, so that a 1024-thread block leaves room for the
// deferred solution update (k_update_x, one 128-thread block per SM) beside it; the FP64 tiles
// (256 threads) need more.
template <class F2, class G, bool POST>
__global__ void __maxnreg__(56) kacz_sweep_tile_kernel(float2* __restrict__ uout, int po,
                                                       const float2* __restrict__ uin, int pu,
                                                       const F2* __restrict__ f, int pf, const float* __restrict__ kh,
                                                       int pk, int n, float bA, const int* __restrict__ stop, Inst bi) {
  tile_sweeps<float, F2, G, POST>(uout, po, uin, pu, f, pf, kh, pk, n, bA, stop, bi);
}
template <class G, bool POST>
__global__ void __launch_bounds__(G::TBK) kacz_sweep_tile64_kernel(double2* __restrict__ uout, int po,
                                                                   const double2* __restrict__ uin, int pu,
                                                                   const double2* __restrict__ f, int pf,
                                                                   const double* __restrict__ kh, int pk, int n,
                                                                   double bA, const int* __restrict__ stop, Inst bi) {
  tile_sweeps<double, double2, G, POST>(uout, po, uin, pu, f, pf, kh, pk, n, bA, stop, bi);
}
template <class T, class F2, class G, bool POST>
struct TileKernel {
  static constexpr auto fn = kacz_sweep_tile_kernel<F2, G, POST>;
};
template <class G, bool POST>
struct TileKernel<double, double2, G, POST> {
  static constexpr auto fn = kacz_sweep_tile64_kernel<G, POST>;
};

template <class T>
size_t level_smem(int n) {
  return (size_t)lvl::blocked_cells(n) * (3 * sizeof(c2<T>) + sizeof(T));
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

// ------------------------------------------------------------------ whole level in a cluster
// The level's rows are split into bands over the C blocks of a thread-block cluster (C <= 16),
// each block holding its band of u, f~, the row diagonals and 1/|a_p|^2 in shared memory. A row
// action on a band's first or last row reads and updates one node of the neighbouring band
// through distributed shared memory; rows of one colour have disjoint supports, so no node is
// touched twice in a colour, and a cluster barrier separates the colours. Same operations as the
// one-block form (hz_level.cuh), spread over C SMs: for the FP64 form this is C times the FP64
// rate of one SM on the Kaczmarz level.
namespace {

namespace cgx = cooperative_groups;
constexpr int KC_THREADS = 256;

template <class T>
struct ClusterLevel {
  c2<T>* su;   // [band][w]
  c2<T>* sf;
  c2<T>* sd;
  T* sinv;
  c2<T>* sr;   // residual (pre), in place of the diagonals once the sweeps are done
  int w, n, rows, r0, r1;  // band rows [r0, r1), rows per band
  __device__ ClusterLevel(unsigned char* smem, int n_, int rows_, int rank) {
    n = n_;
    w = n + 1;
    rows = rows_;
    r0 = min(rank * rows, n + 1);
    r1 = min(r0 + rows, w);
    const int cells = rows * w;
    su = reinterpret_cast<c2<T>*>(smem);
    sf = su + cells;
    sd = sf + cells;
    sr = sd;
    sinv = reinterpret_cast<T*>(sd + cells);
  }
  // row j of array a (one of su, sr), in whichever block of the cluster owns it
  __device__ c2<T>* row(cgx::cluster_group& cl, c2<T>* a, int j) const {
    const int owner = j / rows;
    c2<T>* base = cl.map_shared_rank(a, owner);
    return base + (j - owner * rows) * w;
  }
};

template <class T>
__device__ __forceinline__ void cluster_act(cgx::cluster_group& cl, const ClusterLevel<T>& L, int i, int j) {
  const int n = L.n;
  const int lr = j - L.r0;
  c2<T>* rp = L.su + lr * L.w;
  const int jS = j > 0 ? j - 1 : 1, jN = j < n ? j + 1 : n - 1;
  c2<T>* rs = (jS >= L.r0 && jS < L.r1) ? L.su + (jS - L.r0) * L.w : L.row(cl, L.su, jS);
  c2<T>* rn = (jN >= L.r0 && jN < L.r1) ? L.su + (jN - L.r0) * L.w : L.row(cl, L.su, jN);
  const int iW = i > 0 ? i - 1 : 1, iE = i < n ? i + 1 : n - 1;
  const int p = lr * L.w + i;
  lvl::act_nodes<T>(rp + i, rp + iW, rp + iE, rs + i, rn + i, L.sf[p], L.sd[p], L.sinv[p]);
}

template <class T>
__device__ void cluster_sweeps(cgx::cluster_group& cl, const ClusterLevel<T>& L, int nu, bool post) {
  const int M = (L.w + 4) / 5, nrow = L.r1 - L.r0;
  for (int s = 0; s < nu; ++s)
    for (int k = 0; k < 5; ++k) {
      const int colour = post ? 4 - k : k;
      for (int t = threadIdx.x; t < nrow * M; t += blockDim.x) {
        const int jl = t / M, m = t - jl * M, j = L.r0 + jl;
        int i0 = colour + (3 * j) % 5;
        i0 = i0 >= 5 ? i0 - 5 : i0;
        const int i = i0 + 5 * m;
        if (i <= L.n) cluster_act<T>(cl, L, i, j);
      }
      cl.sync();
    }
}

template <class T>
__global__ void __launch_bounds__(KC_THREADS) kacz_cluster_pre_kernel(c2<T>* __restrict__ u, int pu,
                                                                       c2<T>* __restrict__ fc, int pc,
                                                                       const c2<T>* __restrict__ f, int pf,
                                                                       const T* __restrict__ kh, int pk, int n, T bA,
                                                                       T bB, int nu, int rows,
                                                                       const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;  // the whole cluster (one instance) returns
  cgx::cluster_group cl = cgx::this_cluster();
  u += blockIdx.z * bi.su;
  fc += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  const ClusterLevel<T> L(smem, n, rows, (int)cl.block_rank());
  const int w = L.w, cells = (L.r1 - L.r0) * w;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    const int j = L.r0 + q / w, i = q % w;
    L.su[q] = mk<T>(0, 0);
    L.sf[q] = f[(long long)j * pf + i];
    lvl::row_consts<T>(kh[(long long)j * pk + i], i, j, n, bA, &L.sd[q], &L.sinv[q]);
  }
  cl.sync();
  cluster_sweeps<T>(cl, L, nu, false);
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    const int j = L.r0 + q / w, i = q % w;
    u[(long long)j * pu + i] = L.su[q];
    const int jS = j > 0 ? j - 1 : 1, jN = j < n ? j + 1 : n - 1;
    const int iW = i > 0 ? i - 1 : 1, iE = i < n ? i + 1 : n - 1;
    const c2<T>* rs = L.row(cl, L.su, jS);
    const c2<T>* rn = L.row(cl, L.su, jN);
    const c2<T>* rp = L.su + (j - L.r0) * w;
    const c2<T> nb = xr::nb4<T>(rp[iW], rp[iE], rs[i], rn[i]);
    L.sr[q] = xr::resid<T>(L.sf[q], L.su[q], nb, xr::diag<T>(kh[(long long)j * pk + i], lvl::sides_at(i, j, n), bB));
  }
  cl.sync();
  // full weighting of the coarse rows whose centre row lies in this band
  const int wc = n / 2 + 1, J0 = (L.r0 + 1) / 2, J1 = min((L.r1 + 1) / 2, wc);  // 2J in [r0, r1)
  for (int q = threadIdx.x; q < (J1 - J0) * wc; q += blockDim.x) {
    const int J = J0 + q / wc, I = q % wc;
    c2<T> rowsum[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const c2<T>* rr = L.row(cl, L.sr, reflect(2 * J + b - 1, n));
      rowsum[b] = xr::fw3<T>(rr[reflect(2 * I - 1, n)], rr[2 * I], rr[reflect(2 * I + 1, n)]);
    }
    fc[(long long)J * pc + I] = xr::cscale<T>(xr::fw3<T>(rowsum[0], rowsum[1], rowsum[2]), (T)0.25);
  }
  cl.sync();  // no block leaves while others may still read its shared memory
}

template <class T>
__global__ void __launch_bounds__(KC_THREADS) kacz_cluster_post_kernel(c2<T>* __restrict__ u, int pu,
                                                                        const c2<T>* __restrict__ ec, int pc,
                                                                        const c2<T>* __restrict__ f, int pf,
                                                                        const T* __restrict__ kh, int pk, int n, T bA,
                                                                        int nu, int rows, const int* __restrict__ stop,
                                                                        Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  cgx::cluster_group cl = cgx::this_cluster();
  u += blockIdx.z * bi.su;
  ec += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  const ClusterLevel<T> L(smem, n, rows, (int)cl.block_rank());
  const int w = L.w, cells = (L.r1 - L.r0) * w;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    const int j = L.r0 + q / w, i = q % w;
    const c2<T>* e0 = ec + (long long)(j >> 1) * pc;
    L.su[q] = xr::cadd<T>(u[(long long)j * pu + i], xr::bilinear<T>(e0, e0 + pc, i >> 1, i & 1, j & 1));
    L.sf[q] = f[(long long)j * pf + i];
    lvl::row_consts<T>(kh[(long long)j * pk + i], i, j, n, bA, &L.sd[q], &L.sinv[q]);
  }
  cl.sync();
  cluster_sweeps<T>(cl, L, nu, true);
  for (int q = threadIdx.x; q < cells; q += blockDim.x) u[(long long)(L.r0 + q / w) * pu + q % w] = L.su[q];
  cl.sync();
}

template <class T>
size_t cluster_smem(int n, int rows) {
  return (size_t)rows * (n + 1) * (3 * sizeof(c2<T>) + sizeof(T));
}

template <class T>
cudaError_t cluster_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kacz_cluster_pre_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       KACZ_LEVEL_MAX_SMEM);
  if (!e) e = cudaFuncSetAttribute(kacz_cluster_post_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   KACZ_LEVEL_MAX_SMEM);
  if (!e) e = cudaFuncSetAttribute(kacz_cluster_pre_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (!e) e = cudaFuncSetAttribute(kacz_cluster_post_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (!e) done = true;
  return e;
}

template <class T, class... Args>
cudaError_t launch_cluster_kernel(void (*kernel)(Args...), int c, size_t smem, cudaStream_t s, const Inst& bi,
                                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c, 1, bi.count);
  cfg.blockDim = dim3(KC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

template <class T, class F2, class G, bool POST>
cudaError_t tile_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(TileKernel<T, F2, G, POST>::fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tile_smem<T, G>());
  if (!e) done = true;
  return e;
}

template <class T, class F2, class G>
cudaError_t tile_launch(void* uout, int po, const void* uin, int pu, const void* f, int pf, const void* kh, int pk,
                        int n, double bA, bool post, const int* stop, cudaStream_t s, const Inst& bi) {
  cudaError_t e = post ? tile_attr<T, F2, G, true>() : tile_attr<T, F2, G, false>();
  if (e) return e;
  dim3 grid((n + G::KT) / G::KT, (n + G::KT) / G::KT, bi.count);
  if (post)
    pdl_launch(TileKernel<T, F2, G, true>::fn, grid, G::TBK, tile_smem<T, G>(), s, (c2<T>*)uout, po,
               (const c2<T>*)uin, pu, (const F2*)f, pf, (const T*)kh, pk, n, (T)bA, stop, bi);
  else
    pdl_launch(TileKernel<T, F2, G, false>::fn, grid, G::TBK, tile_smem<T, G>(), s, (c2<T>*)uout, po,
               (const c2<T>*)uin, pu, (const F2*)f, pf, (const T*)kh, pk, n, (T)bA, stop, bi);
  return cudaGetLastError();
}

int kacz_tile_sweeps_per_launch(bool fp32, int n, int nu) {
  // two sweeps per launch on FP32 levels of at least 256 intervals: with the two-sweep halo,
  // 64-node tiles (n_l >= 1024) read 1.03 region nodes per output and sweep and 32-node tiles
  // (n_l = 256 .. 1023, where 64-node tiles are too few to fill the GPU) 1.75, against 2.06 for
  // one sweep on 32-node tiles. The launches ping-pong between two arrays and must end in u from an
  // input in u, so their number has to be even: nu a multiple of 4.
  return (fp32 && n >= 256 && nu % 4 == 0) ? 2 : 1;
}

cudaError_t launch_kacz_sweep_tile(bool fp32, void* uout, int po, const void* uin, int pu, const void* f, int pf,
                                   bool f64_src, const void* kh, int pk, int n, double bA, bool post, int sweeps,
                                   const int* stop, cudaStream_t s, const Inst& bi) {
  if (!fp32)
    return tile_launch<double, double2, TileOne>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi);
  if (sweeps == 2 && n >= 1024)
    return f64_src ? tile_launch<float, double2, TileTwo>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi)
                   : tile_launch<float, float2, TileTwo>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi);
  if (sweeps == 2)
    return f64_src ? tile_launch<float, double2, TileTwoS>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi)
                   : tile_launch<float, float2, TileTwoS>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi);
  return f64_src ? tile_launch<float, double2, TileOne>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi)
                 : tile_launch<float, float2, TileOne>(uout, po, uin, pu, f, pf, kh, pk, n, bA, post, stop, s, bi);
}

namespace {

// Cluster shape of a level: the most blocks (16, 8, 4 or 2; 16 is beyond the portable cluster
// size) whose bands fit KACZ_LEVEL_MAX_SMEM and that the device can co-schedule, found once per
// (precision, n). c = 0: no cluster form for this level.
struct ClusterShape {
  int c = 0, rows = 0;
  size_t smem = 0;
};
template <class T>
ClusterShape cluster_shape(int n) {
  static std::mutex mu;
  static std::map<int, ClusterShape> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(n);
  if (it != cache.end()) return it->second;
  ClusterShape best;
  if (!cluster_attr<T>()) {
    for (int c = 16; c >= 2 && !best.c; c /= 2) {
      const int rows = (n + 1 + c - 1) / c;
      const size_t smem = cluster_smem<T>(n, rows);
      if (smem > (size_t)KACZ_LEVEL_MAX_SMEM) break;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(KC_THREADS);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = c;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int active = 0;
      if (cudaOccupancyMaxActiveClusters(&active, kacz_cluster_pre_kernel<T>, &cfg) == cudaSuccess && active > 0 &&
          cudaOccupancyMaxActiveClusters(&active, kacz_cluster_post_kernel<T>, &cfg) == cudaSuccess && active > 0)
        best = ClusterShape{c, rows, smem};
    }
    cudaGetLastError();  // an unsupported shape leaves no sticky error
  }
  cache[n] = best;
  return best;
}

}  // namespace

bool kacz_cluster_fits(bool fp32, int n) { return (fp32 ? cluster_shape<float>(n) : cluster_shape<double>(n)).c > 0; }

cudaError_t launch_kacz_cluster_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                    int pk, int n, double bA, double bB, int nu, const int* stop, cudaStream_t s,
                                    const Inst& bi) {
  cudaError_t e;
  if (fp32) {
    const ClusterShape C = cluster_shape<float>(n);
    if (!C.c) return cudaErrorInvalidValue;
    e = launch_cluster_kernel<float>(kacz_cluster_pre_kernel<float>, C.c, C.smem, s, bi, (float2*)u, pu, (float2*)fc,
                                     pc, (const float2*)f, pf, (const float*)kh, pk, n, (float)bA, (float)bB, nu, C.rows,
                                     stop, bi);
  } else {
    const ClusterShape C = cluster_shape<double>(n);
    if (!C.c) return cudaErrorInvalidValue;
    e = launch_cluster_kernel<double>(kacz_cluster_pre_kernel<double>, C.c, C.smem, s, bi, (double2*)u, pu,
                                      (double2*)fc, pc, (const double2*)f, pf, (const double*)kh, pk, n, bA, bB, nu,
                                      C.rows, stop, bi);
  }
  return e ? e : cudaGetLastError();
}

cudaError_t launch_kacz_cluster_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                     const void* kh, int pk, int n, double bA, int nu, const int* stop, cudaStream_t s,
                                     const Inst& bi) {
  cudaError_t e;
  if (fp32) {
    const ClusterShape C = cluster_shape<float>(n);
    if (!C.c) return cudaErrorInvalidValue;
    e = launch_cluster_kernel<float>(kacz_cluster_post_kernel<float>, C.c, C.smem, s, bi, (float2*)u, pu,
                                     (const float2*)ec, pc, (const float2*)f, pf, (const float*)kh, pk, n, (float)bA,
                                     nu, C.rows, stop, bi);
  } else {
    const ClusterShape C = cluster_shape<double>(n);
    if (!C.c) return cudaErrorInvalidValue;
    e = launch_cluster_kernel<double>(kacz_cluster_post_kernel<double>, C.c, C.smem, s, bi, (double2*)u, pu,
                                      (const double2*)ec, pc, (const double2*)f, pf, (const double*)kh, pk, n, bA, nu,
                                      C.rows, stop, bi);
  }
  return e ? e : cudaGetLastError();
}

}  // namespace hz
