// Whole-level operations on a small grid held in one block's shared memory (row pitch n + 1):
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

// Row action on row (i, j) of a level stored whole with row pitch w.
template <class T>
__device__ __forceinline__ void act(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int w, int i, int j,
                                    int n) {
  const int p = j * w + i;
  act_at<T>(su, sf[p], sd[p], sinv[p], p, i > 0 ? -1 : 1, i < n ? 1 : -1, j > 0 ? -w : w, j < n ? w : -w);
}

// Thread -> row of a colour (i + 2j) mod 5: grid row j holds the colour at i = i0(j) + 5m,
// m < M = ceil((n+1)/5), i0 = (colour + 3j) mod 5; slot t is (j, m) = (t / M, t % M). Rows of one
// colour have disjoint supports, so a colour is one set of independent row actions.
struct ColourSlot {
  int j, m, b;  // b = 3j mod 5
};
__device__ __forceinline__ ColourSlot colour_slot(int t, int M) {
  ColourSlot c;
  c.j = t / M;
  c.m = t - c.j * M;
  c.b = (3 * c.j) % 5;
  return c;
}
template <class T>
__device__ __forceinline__ void act_slot(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int n,
                                         int colour, const ColourSlot& cs) {
  int i0 = colour + cs.b;
  i0 = i0 >= 5 ? i0 - 5 : i0;
  const int i = i0 + 5 * cs.m;
  if (i > n || cs.j > n) return;
  act<T>(su, sf, sd, sinv, n + 1, i, cs.j, n);
}

// nu Kaczmarz sweeps over the colours 0..4 (or 4..0 when `post`), a barrier after each colour.
template <class T>
__device__ __forceinline__ void kacz_sweeps(c2<T>* su, const c2<T>* sf, const c2<T>* sd, const T* sinv, int n, int nu,
                                            bool post) {
  const int w = n + 1, M = (w + 4) / 5;
  if (w * M <= (int)blockDim.x) {
    const ColourSlot cs = colour_slot(threadIdx.x, M);
    for (int s = 0; s < nu; ++s)
      for (int k = 0; k < 5; ++k) {
        act_slot<T>(su, sf, sd, sinv, n, post ? 4 - k : k, cs);
        __syncthreads();
      }
  } else {
    for (int s = 0; s < nu; ++s)
      for (int k = 0; k < 5; ++k) {
        for (int t = threadIdx.x; t < w * M; t += blockDim.x)
          act_slot<T>(su, sf, sd, sinv, n, post ? 4 - k : k, colour_slot(t, M));
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
// r = f~ - B u, with k H from `k` (pitch pk; shared or global).
template <class T>
__device__ __forceinline__ void residual(c2<T>* r, const c2<T>* u, const c2<T>* f, const T* k, int pk, int n, T bB) {
  const int w = n + 1, N = w * w;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int j = q / w, i = q - j * w;
    r[q] = xr::resid<T>(f[q], u[q], nb_at<T>(u, i, j, n), xr::diag<T>(k[(long long)j * pk + i], sides_at(i, j, n), bB));
  }
}
// fc (pitch pc) = full weighting of r onto the (n/2 + 1)^2 grid.
template <class T>
__device__ __forceinline__ void restrict_fw(c2<T>* fc, int pc, const c2<T>* r, int n) {
  const int wc = n / 2 + 1;
  for (int q = threadIdx.x; q < wc * wc; q += blockDim.x) {
    const int J = q / wc, I = q - J * wc;
    fc[(long long)J * pc + I] = xr::fw_node<T>(r, n + 1, n, I, J);
  }
}
// u += P e (e: (n/2 + 1)^2 grid, pitch pe).
template <class T>
__device__ __forceinline__ void prolong_add(c2<T>* u, const c2<T>* e, int pe, int n) {
  const int w = n + 1, N = w * w;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int j = q / w, i = q - j * w;
    const c2<T>* e0 = e + (long long)(j >> 1) * pe;
    u[q] = xr::cadd<T>(u[q], xr::bilinear<T>(e0, e0 + pe, i >> 1, i & 1, j & 1));
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
