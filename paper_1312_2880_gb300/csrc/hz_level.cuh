// Whole-level operations on a small grid held in one block's shared memory (row-major storage,
// or colour-blocked for Kaczmarz levels):
// Kaczmarz row actions over the five colours, one red-black Gauss-Seidel sweep each way, the
// residual, full weighting, bilinear correction and the coarsest dense solve. They run with all
// threads of the block striding over the nodes and a barrier between dependent phases, and use
// the fixed-rounding helpers (xr::), so a level relaxed here gives the same bits as the same
// level relaxed by the tiled or streaming kernels.
#pragma once

#include "hz_common.cuh"

namespace hz {
namespace lvl {

__device__ __forceinline__ int sides_at(int i, int j, int n) { return (i == 0) + (i == n) + (j == 0) + (j == n); }

// ------------------------------------------------------------------ storage of a level
// Natural: row-major with pitch w. Blocked (Kaczmarz levels): the five nodes i = 5m .. 5m + 4 of
// grid row j form slot t = j M + m (M = ceil(w / 5)) of five cells, each node in the cell of its
// colour c = (i + 2j) mod 5: node (i, j) at 5 (j M + i div 5) + (i + 2j) mod 5; 5 w M >= w^2
// cells hold the level. In a colour phase thread t acts on the node of that colour in slot t:
// consecutive threads touch cells 5 apart (no shared-memory bank conflicts, where row-major
// storage cost ~1.7 extra wavefronts per access), and the neighbours lie at fixed cell offsets
// from the slot, so a phase needs almost no index arithmetic.
struct Natural {
  static constexpr bool blocked = false;
  int w;
  __device__ __forceinline__ int at(int i, int j) const { return j * w + i; }
};
struct Blocked {
  static constexpr bool blocked = true;
  int M;
  __device__ __forceinline__ int at(int i, int j) const { return 5 * (j * M + i / 5) + (i + 2 * j) % 5; }
};
__host__ __device__ __forceinline__ int blocked_cols(int n) { return (n + 5) / 5; }
__host__ __device__ __forceinline__ int blocked_cells(int n) { return 5 * (n + 1) * blocked_cols(n); }
__device__ __forceinline__ Blocked blocked(int n) { return Blocked{blocked_cols(n)}; }

// Asynchronous global -> shared copy of one element of B = 4, 8 or 16 bytes (cp.async); the
// copies in flight complete at cp_async_wait_all.
template <int B>
__device__ __forceinline__ void cp_async(void* dst_smem, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else if constexpr (B == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Calls fn(q, i, j) for q = threadIdx.x, threadIdx.x + blockDim.x, ... < count with
// (i, j) = (q mod w, q div w), advanced without a division per step. Threads without a node
// leave at once: on the small levels most warps of the block have none, and their setup would
// otherwise take issue slots from the warps that do.
template <class F>
__device__ __forceinline__ void for_nodes(int w, int count, F&& fn) {
  if ((int)threadIdx.x >= count) return;
  const int step = blockDim.x, dj = step / w, di = step - dj * w;
  int j = threadIdx.x / w, i = threadIdx.x - j * w;
  for (int q = threadIdx.x; q < count; q += step) {
    fn(q, i, j);
    i += di;
    j += dj;
    if (i >= w) {
      i -= w;
      ++j;
    }
  }
}

// Calls fn(q, i, j, p) for every node (i, j) of a Blocked level in row-major order (q = j w + i)
// with its cell p: consecutive threads take consecutive nodes of a grid row, so copies between
// row-major global memory and the level's cells are coalesced on the global side (slot order
// puts a warp's accesses 5 nodes apart, one memory transaction per node).
template <class F>
__device__ __forceinline__ void for_nodes_blocked(int n, F&& fn) {
  const Blocked b = blocked(n);
  for_nodes(n + 1, (n + 1) * (n + 1), [&](int q, int i, int j) { fn(q, i, j, b.at(i, j)); });
}

// ------------------------------------------------------------------ Kaczmarz (Sec. 4)
// Row constants: the diagonal d_p of the relaxation operator and 1 / |a_p|^2 (|d_p|^2 plus the
// squared off-diagonal coefficients: 1 each, 2 for a mirror neighbour, so 4 on an edge).
template <class T>
__device__ __forceinline__ void row_consts(T kh, int i, int j, int n, T beta, c2<T>* d, T* inv) {
  *d = xr::diag<T>(kh, sides_at(i, j, n), beta);
  const T cx = (i == 0 || i == n) ? (T)4 : (T)2, cy = (j == 0 || j == n) ? (T)4 : (T)2;
  *inv = xr::rcp(xr::add(xr::cabs2<T>(*d), cx + cy));
}

// Row action u += conj(a_p) (f_p - a_p u) / |a_p|^2 on the node at up with its neighbours at
// uw, ue, us, un (a mirror neighbour across the boundary is the same node on both sides, so its
// two pointers coincide and it receives 2 delta in one update). The five values are read once and
// written once. Every Kaczmarz kernel form goes through this function, so they give the same bits.
// The arithmetic on the five values already read (mx / my: the W and E, or S and N, support nodes
// are one mirror node, held in uw / us); act_nodes and the two-action form of the tiled sweep call it.
template <class T>
__device__ __forceinline__ void act_update(c2<T>& up, c2<T>& uw, c2<T>& ue, c2<T>& us, c2<T>& un, c2<T> f, c2<T> d,
                                           T inv, bool mx, bool my) {
  const c2<T> delta = xr::cscale<T>(xr::resid<T>(f, up, xr::nb4<T>(uw, ue, us, un), d), inv);
  up = xr::cadd<T>(up, xr::cmulc<T>(d, delta));
  if (mx) {
    uw = xr::cadd<T>(uw, xr::cscale<T>(delta, (T)2));
  } else {
    uw = xr::cadd<T>(uw, delta);
    ue = xr::cadd<T>(ue, delta);
  }
  if (my) {
    us = xr::cadd<T>(us, xr::cscale<T>(delta, (T)2));
  } else {
    us = xr::cadd<T>(us, delta);
    un = xr::cadd<T>(un, delta);
  }
}
template <class T>
__device__ __forceinline__ void act_nodes(c2<T>* pp, c2<T>* pw, c2<T>* pe, c2<T>* ps, c2<T>* pn, c2<T> f, c2<T> d,
                                          T inv) {
  c2<T> up = *pp, uw = *pw, ue = *pe, us = *ps, un = *pn;
  const bool mx = pw == pe, my = ps == pn;
  act_update<T>(up, uw, ue, us, un, f, d, inv, mx, my);
  *pp = up;
  *pw = uw;
  if (!mx) *pe = ue;
  *ps = us;
  if (!my) *pn = un;
}
// The same at shared position p with neighbour offsets dw, de, ds, dn.
template <class T>
__device__ __forceinline__ void act_at(c2<T>* su, c2<T> f, c2<T> d, T inv, int p, int dw, int de, int ds, int dn) {
  act_nodes<T>(su + p, su + p + dw, su + p + de, su + p + ds, su + p + dn, f, d, inv);
}

// Calls fn(i, j, p) for every node (i, j) of a Blocked level with its cell p, slot by slot: slot
// t = (j, m) holds the nodes i = 5m .. 5m + 4, node i = 5m + r in cell 5t + (r + 2j) mod 5. No
// per-node division or modulo.
template <class F>
__device__ __forceinline__ void for_blocked(int n, F&& fn) {
  const int M = blocked_cols(n), S = (n + 1) * M;
  if ((int)threadIdx.x >= S) return;
  const int dj = blockDim.x / M, dm = blockDim.x - dj * M;
  int j = threadIdx.x / M, m = threadIdx.x - j * M;
  for (int t = threadIdx.x; t < S; t += blockDim.x) {
    int c = (2 * j) % 5;
    for (int i = 5 * m; i <= min(5 * m + 4, n); ++i) {
      fn(i, j, 5 * t + c);
      c = c == 4 ? 0 : c + 1;
    }
    m += dm;
    j += dj;
    if (m >= M) {
      m -= M;
      ++j;
    }
  }
}

// A thread's slot t = (j, m) of a Blocked Kaczmarz level: the first cell of the slot (o = 5t) and
// of the slots one grid row down and up (for j = 0 and j = n the mirror row 1 or n - 1 stands in
// for the missing one), and b = 3j mod 5 (the node of colour c in the slot is
// i = 5m + (c + b) mod 5).
struct KaczSlot {
  int o, os, on, m, b, n;
  bool j0, jn;
};
__device__ __forceinline__ KaczSlot kacz_slot(int n, int t) {
  const int M = blocked_cols(n), j = t / M;
  KaczSlot s;
  s.o = 5 * t;
  s.on = 5 * (j < n ? t + M : t - M);
  s.os = 5 * (j > 0 ? t - M : t + M);
  s.m = t - j * M;
  s.b = (3 * j) % 5;
  s.n = n;
  s.j0 = j == 0;
  s.jn = j == n;
  return s;
}
// Cell offsets of colour c's neighbours within a slot: west c - 1, east c + 1, south c - 2,
// north c + 2 (mod 5), the same for every thread of a phase.
struct ColourOffsets {
  int c, cw, ce, cs, cn;
  __device__ __forceinline__ explicit ColourOffsets(int c_)
      : c(c_), cw(c_ == 0 ? 4 : c_ - 1), ce(c_ == 4 ? 0 : c_ + 1), cs(c_ >= 2 ? c_ - 2 : c_ + 3),
        cn(c_ <= 2 ? c_ + 2 : c_ - 3) {}
};
// Row action of colour k.c in slot s: the west neighbour lies in the slot before when the node
// starts its block, the east one in the next slot when it ends it, south and north one grid row
// away; at the boundary the mirror neighbour is the node on the other side.
template <class T>
__device__ __forceinline__ void act_slot(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv,
                                         const KaczSlot& s, const ColourOffsets& k) {
  int i0 = k.c + s.b;
  i0 = i0 >= 5 ? i0 - 5 : i0;
  const int i = i0 + 5 * s.m;
  if (i > s.n) return;
  const int w = s.o + k.cw - (i0 == 0 ? 5 : 0), e = s.o + k.ce + (i0 == 4 ? 5 : 0);
  const int so = s.j0 ? s.on + k.cn : s.os + k.cs, no = s.jn ? s.os + k.cs : s.on + k.cn;
  const int p = s.o + k.c;
  act_nodes<T>(su + p, su + (i == 0 ? e : w), su + (i == s.n ? w : e), su + so, su + no, sf[p], sd[p], sinv[p]);
}
// nu Kaczmarz sweeps over the colours 0..4 (or 4..0 when `post`) on a Blocked level, a barrier
// after each colour. Rows of one colour have disjoint supports, so a colour is one set of
// independent row actions.
template <class T>
__device__ __forceinline__ void kacz_sweeps(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int n, int nu,
                                            bool post) {
  const int S = (n + 1) * blocked_cols(n);
  if (S <= (int)blockDim.x) {  // one slot per thread, set up once
    const bool act = threadIdx.x < (unsigned)S;
    const KaczSlot s = kacz_slot(n, act ? threadIdx.x : 0);
#pragma unroll 1
    for (int q = 0; q < 5 * nu; ++q) {
      const int r = q % 5;
      if (act) act_slot<T>(su, sf, sd, sinv, s, ColourOffsets(post ? 4 - r : r));
      __syncthreads();
    }
  } else {
#pragma unroll 1
    for (int q = 0; q < 5 * nu; ++q) {
      const int r = q % 5;
      const ColourOffsets k(post ? 4 - r : r);
      for (int t = threadIdx.x; t < S; t += blockDim.x) act_slot<T>(su, sf, sd, sinv, kacz_slot(n, t), k);
      __syncthreads();
    }
  }
}

// Bilinear interpolation of e (layout le) at fine node (2I + oi, 2J + oj), in the operation order
// of xr::bilinear.
template <class T, class LE>
__device__ __forceinline__ c2<T> bilinear_at(const c2<T>* e, LE le, int I, int J, int oi, int oj) {
  if (oi && oj)
    return xr::cscale<T>(xr::cadd<T>(xr::cadd<T>(e[le.at(I, J)], e[le.at(I, J + 1)]),
                                     xr::cadd<T>(e[le.at(I + 1, J)], e[le.at(I + 1, J + 1)])),
                         (T)0.25);
  if (oi) return xr::cscale<T>(xr::cadd<T>(e[le.at(I, J)], e[le.at(I + 1, J)]), (T)0.5);
  if (oj) return xr::cscale<T>(xr::cadd<T>(e[le.at(I, J)], e[le.at(I, J + 1)]), (T)0.5);
  return e[le.at(I, J)];
}
// ------------------------------------------------------------------ Gauss-Seidel (one sweep)
// The nodes of colour c ((i + j) mod 2 == c): slot q is (j, i) = (q / HW, 2 (q % HW) + (c + j) mod 2).
template <class T, class F>
__device__ __forceinline__ void for_colour(int n, int colour, F&& fn) {
  const int w = n + 1, HW = (w + 1) / 2;
  for_nodes(HW, w * HW, [&](int, int h, int j) {
    const int i = 2 * h + ((colour + j) & 1);
    if (i <= n) fn(i, j);
  });
}
template <class T>
__device__ __forceinline__ c2<T> nb_at(const c2<T>* u, int i, int j, int n) {
  const Nbr b = neighbours(i, j, n);
  const int w = n + 1;
  return xr::nb4<T>(u[j * w + b.iw], u[j * w + b.ie], u[b.js * w + i], u[b.jn * w + i]);
}
// Red node of the pre-sweep from a zero guess: u = f~ / d.
template <class T>
__device__ __forceinline__ c2<T> gs_red_zero(c2<T> f, T k, int i, int j, int n, T bA) {
  return xr::cdiv<T>(f, xr::diag<T>(k, sides_at(i, j, n), bA));
}
// Red nodes from a zero guess, no barrier (the caller's next barrier ends the phase).
template <class T>
__device__ __forceinline__ void gs_red(c2<T>* u, const c2<T>* f, const T* k, int n, T bA) {
  const int w = n + 1;
  for_colour<T>(n, 0, [&](int i, int j) {
    const int p = j * w + i;
    u[p] = gs_red_zero<T>(f[p], k[p], i, j, n, bA);
  });
}
// Black nodes from their red neighbours, then a barrier.
template <class T>
__device__ __forceinline__ void gs_black(c2<T>* u, const c2<T>* f, const T* k, int n, T bA) {
  const int w = n + 1;
  for_colour<T>(n, 1, [&](int i, int j) {
    const int p = j * w + i;
    u[p] = xr::gs<T>(f[p], nb_at<T>(u, i, j, n), xr::diag<T>(k[p], sides_at(i, j, n), bA));
  });
  __syncthreads();
}
// Correction u += P e (e: layout le) and the post-sweep, black nodes then red, in two phases. A
// Gauss-Seidel update does not read the node's own value, so the corrected values are needed
// only at red nodes, as neighbours of the black update: the black phase forms them on the fly
// (the same cadd of u and the bilinear value that a separate correction pass would store) and
// the red phase reads the new black values. Same results as a correction pass followed by the
// black and red updates.
// The red neighbours of a black node are coincident with coarse nodes (both indices even) or at
// coarse cell centres (both odd): on an even row the west and east ones are coincident and the
// south and north ones centres, on an odd row the reverse (mirror neighbours keep the parity, n
// being even). The black nodes of the even rows come first in the walk and those of the odd rows
// after, so a warp rarely mixes the two cases; the corrected values are the ones bilinear_at
// gives (same operations).
template <class T, class LE>
__device__ __forceinline__ void gs_post_corrected(c2<T>* u, const c2<T>* f, const T* k, int n, T bA, const c2<T>* e,
                                                  LE le) {
  const int w = n + 1, HW = (w + 1) / 2, even_slots = (n / 2 + 1) * HW;
  auto coinc = [&](int i, int j) { return xr::cadd<T>(u[j * w + i], e[le.at(i >> 1, j >> 1)]); };
  auto centre = [&](int i, int j) {
    const int I = i >> 1, J = j >> 1;
    return xr::cadd<T>(u[j * w + i], xr::cscale<T>(xr::cadd<T>(xr::cadd<T>(e[le.at(I, J)], e[le.at(I, J + 1)]),
                                                                xr::cadd<T>(e[le.at(I + 1, J)], e[le.at(I + 1, J + 1)])),
                                                    (T)0.25));
  };
  for (int q = threadIdx.x; q < even_slots + (n / 2) * HW; q += blockDim.x) {
    const int odd = q >= even_slots, r = odd ? q - even_slots : q;
    const int jj = r / HW, h = r - jj * HW, j = 2 * jj + odd, i = 2 * h + ((1 + j) & 1);
    if (i > n) continue;
    const Nbr b = neighbours(i, j, n);
    const int p = j * w + i;
    const c2<T> nb = odd ? xr::nb4<T>(centre(b.iw, j), centre(b.ie, j), coinc(i, b.js), coinc(i, b.jn))
                         : xr::nb4<T>(coinc(b.iw, j), coinc(b.ie, j), centre(i, b.js), centre(i, b.jn));
    u[p] = xr::gs<T>(f[p], nb, xr::diag<T>(k[p], sides_at(i, j, n), bA));
  }
  __syncthreads();
  for_colour<T>(n, 0, [&](int i, int j) {
    const int p = j * w + i;
    u[p] = xr::gs<T>(f[p], nb_at<T>(u, i, j, n), xr::diag<T>(k[p], sides_at(i, j, n), bA));
  });
  __syncthreads();
}
// ------------------------------------------------------------------ residual and transfers
// r (natural, pitch n + 1) = f~ - B u, u and f~ stored with layout lu, k H from `k` (pitch pk;
// shared or global).
template <class T, class LU>
__device__ __forceinline__ void residual(c2<T>* r, const c2<T>* u, const c2<T>* f, LU lu, const T* k, int pk, int n,
                                         T bB) {
  const int w = n + 1;
  for_nodes(w, w * w, [&](int q, int i, int j) {
    const Nbr b = neighbours(i, j, n);
    const int p = lu.at(i, j);
    r[q] = xr::resid<T>(f[p], u[p], xr::nb4<T>(u[lu.at(b.iw, j)], u[lu.at(b.ie, j)], u[lu.at(i, b.js)], u[lu.at(i, b.jn)]),
                        xr::diag<T>(k[(long long)j * pk + i], sides_at(i, j, n), bB));
  });
}
// The same residual for u and f~ stored Blocked, visited slot by slot: the neighbours' cells
// follow from the node's colour c and position r = i mod 5 in its slot (west c - 1 in this slot,
// or the one before when r = 0; east c + 1, or the next slot when r = 4; south c - 2 and north
// c + 2 one grid row away), mirrored at the boundary.
template <class T>
__device__ __forceinline__ void residual_blocked(c2<T>* r, const c2<T>* u, const c2<T>* f, const T* k, int pk, int n,
                                                 T bB) {
  const int w = n + 1, M5 = 5 * blocked_cols(n);
  for_blocked(n, [&](int i, int j, int p) {
    const int c = p % 5, t5 = p - c, ri = i % 5;
    const int cw = c == 0 ? 4 : c - 1, ce = c == 4 ? 0 : c + 1, cs = c >= 2 ? c - 2 : c + 3, cn = c <= 2 ? c + 2 : c - 3;
    const int pw = (ri > 0 ? t5 : t5 - 5) + cw, pe = (ri < 4 ? t5 : t5 + 5) + ce;
    const int ps = t5 - M5 + cs, pn = t5 + M5 + cn;
    const int qw = i > 0 ? pw : pe, qe = i < n ? pe : pw, qs = j > 0 ? ps : pn, qn = j < n ? pn : ps;
    r[j * w + i] = xr::resid<T>(f[p], u[p], xr::nb4<T>(u[qw], u[qe], u[qs], u[qn]),
                                xr::diag<T>(k[(long long)j * pk + i], sides_at(i, j, n), bB));
  });
}
// fc (layout lc) = full weighting of r (natural) onto the (n/2 + 1)^2 grid.
// Full weighting onto a row-major Gauss-Seidel level (pitch n/2 + 1), which also starts that
// level's pre-sweep: its red nodes from a zero guess (k H of the coarse level kc, relaxation
// beta bAc) need only their own restricted value.
template <class T>
__device__ __forceinline__ void restrict_fw_red(c2<T>* fc, c2<T>* uc, const T* kc, T bAc, const c2<T>* r, int n) {
  const int nc = n / 2, wc = nc + 1;
  for_nodes(wc, wc * wc, [&](int q, int I, int J) {
    const c2<T> v = xr::fw_node<T>(r, n + 1, n, I, J);
    fc[q] = v;
    if (((I + J) & 1) == 0) uc[q] = gs_red_zero<T>(v, kc[q], I, J, nc, bAc);
  });
}
template <class T, class LC>
__device__ __forceinline__ void restrict_fw(c2<T>* fc, LC lc, const c2<T>* r, int n) {
  const int wc = n / 2 + 1;
  if constexpr (LC::blocked)
    for_blocked(n / 2, [&](int I, int J, int p) { fc[p] = xr::fw_node<T>(r, n + 1, n, I, J); });
  else
    for_nodes(wc, wc * wc, [&](int, int I, int J) { fc[lc.at(I, J)] = xr::fw_node<T>(r, n + 1, n, I, J); });
}
// u (layout lu) += P e (e: (n/2 + 1)^2 grid, layout le).
// On a Blocked level the nodes are walked one parity class (i mod 2, j mod 2) at a time, so the
// threads of a warp take the same interpolation case.
template <class T, class LU, class LE>
__device__ __forceinline__ void prolong_add(c2<T>* u, LU lu, const c2<T>* e, LE le, int n) {
  if constexpr (LU::blocked) {
#pragma unroll
    for (int cls = 0; cls < 4; ++cls) {
      const int oi = cls & 1, oj = cls >> 1, wi = (n - oi) / 2 + 1, wj = (n - oj) / 2 + 1;
      for_nodes(wi, wi * wj, [&](int, int I, int J) {
        const int p = lu.at(2 * I + oi, 2 * J + oj);
        u[p] = xr::cadd<T>(u[p], bilinear_at<T>(e, le, I, J, oi, oj));
      });
    }
  } else {
    for_nodes(n + 1, (n + 1) * (n + 1), [&](int q, int i, int j) {
      u[q] = xr::cadd<T>(u[q], bilinear_at<T>(e, le, i >> 1, j >> 1, i & 1, j & 1));
    });
  }
}
// Row r of the coarsest solve u = A^-1 f (inverse stored transposed, m x m), accumulated in column
// order. The inverse is read from global memory eight columns at a time before they are summed,
// so eight loads are in flight instead of one.
template <class T>
__device__ __forceinline__ c2<T> coarse_row(const c2<T>* __restrict__ ainvT, const c2<T>* f, int m, int r) {
  constexpr int B = 8;
  c2<T> acc = mk<T>(0, 0);
  int c = 0;
  for (; c + B <= m; c += B) {
    c2<T> a[B];
#pragma unroll
    for (int q = 0; q < B; ++q) a[q] = ainvT[(long long)(c + q) * m + r];
#pragma unroll
    for (int q = 0; q < B; ++q) acc = xr::cadd<T>(acc, xr::cmul<T>(a[q], f[c + q]));
  }
  for (; c < m; ++c) acc = xr::cadd<T>(acc, xr::cmul<T>(ainvT[(long long)c * m + r], f[c]));
  return acc;
}

}  // namespace lvl
}  // namespace hz
