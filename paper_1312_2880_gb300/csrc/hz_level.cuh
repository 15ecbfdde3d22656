// Whole-level operations on a small grid held in one block's shared memory (natural row-major
// storage, or colour-planar for Kaczmarz levels):
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
// Natural: row-major with pitch w. Planar (Kaczmarz levels): the nodes of colour
// c = (i + 2j) mod 5 in grid row j are contiguous, at ((c w + j) M + i div 5) with M = ceil(w / 5)
// (node (i, j) has i mod 5 = (c + 3j) mod 5). A colour phase then reads and writes every array
// with unit stride across the threads of a warp instead of stride 5 across grid rows (which cost
// ~1.7 extra shared-memory wavefronts per access), and 5 w M >= w^2 cells hold the level.
struct Natural {
  int w;
  __device__ __forceinline__ int at(int i, int j) const { return j * w + i; }
};
struct Planar {
  int w, M;
  __device__ __forceinline__ int at(int i, int j) const { return (((i + 2 * j) % 5) * w + j) * M + i / 5; }
};
__host__ __device__ __forceinline__ int planar_cols(int n) { return (n + 5) / 5; }
__host__ __device__ __forceinline__ int planar_cells(int n) { return 5 * (n + 1) * planar_cols(n); }
__device__ __forceinline__ Planar planar(int n) { return Planar{n + 1, planar_cols(n)}; }

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
template <class T>
__device__ __forceinline__ void act_nodes(c2<T>* pp, c2<T>* pw, c2<T>* pe, c2<T>* ps, c2<T>* pn, c2<T> f, c2<T> d,
                                          T inv) {
  const c2<T> up = *pp, uw = *pw, ue = *pe, us = *ps, un = *pn;
  const c2<T> delta = xr::cscale<T>(xr::resid<T>(f, up, xr::nb4<T>(uw, ue, us, un), d), inv);
  *pp = xr::cadd<T>(up, xr::cmulc<T>(d, delta));
  if (pw == pe) {
    *pw = xr::cadd<T>(uw, xr::cscale<T>(delta, (T)2));
  } else {
    *pw = xr::cadd<T>(uw, delta);
    *pe = xr::cadd<T>(ue, delta);
  }
  if (ps == pn) {
    *ps = xr::cadd<T>(us, xr::cscale<T>(delta, (T)2));
  } else {
    *ps = xr::cadd<T>(us, delta);
    *pn = xr::cadd<T>(un, delta);
  }
}
// The same at shared position p with neighbour offsets dw, de, ds, dn.
template <class T>
__device__ __forceinline__ void act_at(c2<T>* su, c2<T> f, c2<T> d, T inv, int p, int dw, int de, int ds, int dn) {
  act_nodes<T>(su + p, su + p + dw, su + p + de, su + p + ds, su + p + dn, f, d, inv);
}

// Row action of colour c on a Planar level, thread slot t = (j, m) = (t div M, t mod M): the node
// (i, j) with i = (c + 3j) mod 5 + 5m (b = 3j mod 5), planar index c w M + t. Its west and east
// neighbours have colours c - 1 and c + 1 in the same row (column m, or m -+ 1 where i mod 5 is
// 0 or 4), south and north colours c - 2 and c + 2 in rows j -+ 1, column m; at the boundary the
// mirror neighbour is the node on the other side.
template <class T>
__device__ __forceinline__ void act_planar(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int n, int M,
                                           int c, int t, int j, int m, int b) {
  int i0 = c + b;
  i0 = i0 >= 5 ? i0 - 5 : i0;
  const int i = i0 + 5 * m;
  if (i > n) return;
  const int plane = (n + 1) * M, row = j * M + m;
  const int cw = c == 0 ? 4 : c - 1, ce = c == 4 ? 0 : c + 1, cs = c >= 2 ? c - 2 : c + 3, cn = c <= 2 ? c + 2 : c - 3;
  const int p = c * plane + t;
  const int pw = cw * plane + row - (i0 == 0), pe = ce * plane + row + (i0 == 4);
  const int ps = cs * plane + row - M, pn = cn * plane + row + M;
  act_nodes<T>(su + p, su + (i == 0 ? pe : pw), su + (i == n ? pw : pe), su + (j == 0 ? pn : ps),
               su + (j == n ? ps : pn), sf[p], sd[p], sinv[p]);
}

// nu Kaczmarz sweeps over the colours 0..4 (or 4..0 when `post`) on a Planar level, a barrier
// after each colour. Rows of one colour have disjoint supports, so a colour is one set of
// independent row actions.
template <class T>
__device__ __forceinline__ void kacz_sweeps(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int n, int nu,
                                            bool post) {
  const int M = planar_cols(n), S = (n + 1) * M;
  if (S <= (int)blockDim.x) {
    const int t = threadIdx.x, j = t / M, m = t - j * M, b = (3 * j) % 5;
    for (int s = 0; s < nu; ++s)
      for (int k = 0; k < 5; ++k) {
        if (t < S) act_planar<T>(su, sf, sd, sinv, n, M, post ? 4 - k : k, t, j, m, b);
        __syncthreads();
      }
  } else {
    for (int s = 0; s < nu; ++s)
      for (int k = 0; k < 5; ++k) {
        for (int t = threadIdx.x; t < S; t += blockDim.x) {
          const int j = t / M;
          act_planar<T>(su, sf, sd, sinv, n, M, post ? 4 - k : k, t, j, t - j * M, (3 * j) % 5);
        }
        __syncthreads();
      }
  }
}

// ------------------------------------------------------------------ Gauss-Seidel (one sweep)
// The nodes of colour c ((i + j) mod 2 == c): slot q is (j, i) = (q / HW, 2 (q % HW) + (c + j) mod 2).
template <class T, class F>
__device__ __forceinline__ void for_colour(int n, int colour, F&& fn) {
  const int w = n + 1, HW = (w + 1) / 2;
  for (int q = threadIdx.x; q < w * HW; q += blockDim.x) {
    const int j = q / HW, i = 2 * (q - j * HW) + ((colour + j) & 1);
    if (i <= n) fn(i, j);
  }
}
template <class T>
__device__ __forceinline__ c2<T> nb_at(const c2<T>* u, int i, int j, int n) {
  const Nbr b = neighbours(i, j, n);
  const int w = n + 1;
  return xr::nb4<T>(u[j * w + b.iw], u[j * w + b.ie], u[b.js * w + i], u[b.jn * w + i]);
}
// Red nodes from a zero guess (u = f~ / d), then black nodes.
template <class T>
__device__ __forceinline__ void gs_pre(c2<T>* u, const c2<T>* f, const T* k, int n, T bA) {
  const int w = n + 1;
  for_colour<T>(n, 0, [&](int i, int j) {
    const int p = j * w + i;
    u[p] = xr::cdiv<T>(f[p], xr::diag<T>(k[p], sides_at(i, j, n), bA));
  });
  __syncthreads();
  for_colour<T>(n, 1, [&](int i, int j) {
    const int p = j * w + i;
    u[p] = xr::gs<T>(f[p], nb_at<T>(u, i, j, n), xr::diag<T>(k[p], sides_at(i, j, n), bA));
  });
  __syncthreads();
}
// Black nodes, then red nodes (the post-sweep on u + P e).
template <class T>
__device__ __forceinline__ void gs_post(c2<T>* u, const c2<T>* f, const T* k, int n, T bA) {
  const int w = n + 1;
#pragma unroll 1
  for (int c = 1; c >= 0; --c) {
    for_colour<T>(n, c, [&](int i, int j) {
      const int p = j * w + i;
      u[p] = xr::gs<T>(f[p], nb_at<T>(u, i, j, n), xr::diag<T>(k[p], sides_at(i, j, n), bA));
    });
    __syncthreads();
  }
}

// ------------------------------------------------------------------ residual and transfers
// r (natural, pitch n + 1) = f~ - B u, u and f~ stored with layout lu, k H from `k` (pitch pk;
// shared or global).
template <class T, class LU>
__device__ __forceinline__ void residual(c2<T>* r, const c2<T>* u, const c2<T>* f, LU lu, const T* k, int pk, int n,
                                         T bB) {
  const int w = n + 1, N = w * w;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int j = q / w, i = q - j * w;
    const Nbr b = neighbours(i, j, n);
    const int p = lu.at(i, j);
    r[q] = xr::resid<T>(f[p], u[p], xr::nb4<T>(u[lu.at(b.iw, j)], u[lu.at(b.ie, j)], u[lu.at(i, b.js)], u[lu.at(i, b.jn)]),
                        xr::diag<T>(k[(long long)j * pk + i], sides_at(i, j, n), bB));
  }
}
// fc (layout lc) = full weighting of r (natural) onto the (n/2 + 1)^2 grid.
template <class T, class LC>
__device__ __forceinline__ void restrict_fw(c2<T>* fc, LC lc, const c2<T>* r, int n) {
  const int wc = n / 2 + 1;
  for (int q = threadIdx.x; q < wc * wc; q += blockDim.x) {
    const int J = q / wc, I = q - J * wc;
    fc[lc.at(I, J)] = xr::fw_node<T>(r, n + 1, n, I, J);
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
// u (layout lu) += P e (e: (n/2 + 1)^2 grid, layout le).
template <class T, class LU, class LE>
__device__ __forceinline__ void prolong_add(c2<T>* u, LU lu, const c2<T>* e, LE le, int n) {
  const int w = n + 1, N = w * w;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int j = q / w, i = q - j * w;
    const int p = lu.at(i, j);
    u[p] = xr::cadd<T>(u[p], bilinear_at<T>(e, le, i >> 1, j >> 1, i & 1, j & 1));
  }
}
// Row r of the coarsest solve u = A^-1 f (inverse stored transposed, m x m).
template <class T>
__device__ __forceinline__ c2<T> coarse_row(const c2<T>* __restrict__ ainvT, const c2<T>* f, int m, int r) {
  c2<T> acc = mk<T>(0, 0);
  for (int c = 0; c < m; ++c) acc = xr::cadd<T>(acc, xr::cmul<T>(ainvT[(long long)c * m + r], f[c]));
  return acc;
}

}  // namespace lvl
}  // namespace hz
