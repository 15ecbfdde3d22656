// Single-node operations of a level held in global memory (row-major, pitch in elements): one
// Kaczmarz row action, the restricted residual of one coarse node, and the bilinear correction of
// one fine node. The per-launch kernels (one colour or one transfer per launch) and the persistent
// grid-synchronised Kaczmarz form both call these, so the two give the same bits.
#pragma once

#include "hz_common.cuh"
#include "hz_level.cuh"

namespace hz {
namespace gnode {

// Row action on row (i, j) of A u = f~ (Sec. 4-5, Kaczmarz): delta = (f~_p - a_p u) / |a_p|^2,
// u_q += conj(a_pq) delta over the row's support (lvl::act_nodes); a mirror neighbour at the
// boundary carries coefficient 2 and receives 2 delta.
template <class T, class F2>
__device__ __forceinline__ void kacz_row(c2<T>* __restrict__ u, int pu, const F2* __restrict__ f, int pf,
                                         const T* __restrict__ kh, int pk, int n, int i, int j, T beta) {
  const Nbr b = neighbours(i, j, n);
  c2<T> d;
  T inv;
  lvl::row_consts<T>(kh[(long long)j * pk + i], i, j, n, beta, &d, &inv);
  c2<T>* row = u + (long long)j * pu;
  lvl::act_nodes<T>(row + i, row + b.iw, row + b.ie, u + (long long)b.js * pu + i, u + (long long)b.jn * pu + i,
                    ldc<T>(f, (long long)j * pf + i), d, inv);
}

// 4 * FW(f~ - B u) at coarse node (I, J): full weighting 1/16 [1 2 1; 2 4 2; 1 2 1] of the fine
// residual around fine node (2I, 2J), fine nodes outside the square mirrored inside; the factor
// 4 = (2H)^2 / H^2 moves it to the coarse level's scaling. The same operations and order as the
// whole-level forms (lvl::residual, xr::fw_node). u is deliberately not __restrict__: in the
// grid-synchronised form other blocks wrote u earlier in the same launch, and a const __restrict__
// pointer lets the compiler read it through the non-coherent read-only path, which may return
// lines cached before those writes.
template <class T, class F2>
__device__ __forceinline__ c2<T> restrict_node(const c2<T>* u, int pu, const F2* __restrict__ f, int pf,
                                               const T* __restrict__ kh, int pk, int n, T beta, int I, int J) {
  c2<T> rows[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int j = reflect(2 * J + b - 1, n);
    c2<T> r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int i = reflect(2 * I + a - 1, n);
      const Nbr nb = neighbours(i, j, n);
      const c2<T>* row = u + (long long)j * pu;
      r[a] = xr::resid<T>(ldc<T>(f, (long long)j * pf + i), row[i],
                          xr::nb4<T>(row[nb.iw], row[nb.ie], u[(long long)nb.js * pu + i], u[(long long)nb.jn * pu + i]),
                          xr::diag<T>(kh[(long long)j * pk + i], lvl::sides_at(i, j, n), beta));
    }
    rows[b] = xr::fw3<T>(r[0], r[1], r[2]);
  }
  return xr::cscale<T>(xr::fw3<T>(rows[0], rows[1], rows[2]), (T)0.25);
}

// u(i, j) += (P e_c)(i, j), bilinear interpolation from the (n/2+1)^2 grid.
template <class T>
__device__ __forceinline__ void prolong_add_node(c2<T>* __restrict__ u, int pu, const c2<T>* __restrict__ ec, int pc,
                                                 int i, int j) {
  const c2<T>* e0 = ec + (long long)(j >> 1) * pc;
  const long long p = (long long)j * pu + i;
  u[p] = xr::cadd<T>(u[p], xr::bilinear<T>(e0, e0 + pc, i >> 1, i & 1, j & 1));
}

}  // namespace gnode
}  // namespace hz
