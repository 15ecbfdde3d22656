// The coarse tail of the V-cycle (Sec. 5) in one block: every level from the first one that fits
// down to the coarsest is held in shared memory, and one launch runs its pre-relaxation and
// restriction on the way down, the dense coarsest solve, and the correction and post-relaxation
// on the way up. Below a few thousand nodes a level's kernels are bound by launch and ramp
// latency, not by work, so this replaces 2 (L - lt) - 1 launches by one. Each level's operations
// are the ones the per-level kernels perform (hz_level.cuh, fixed-rounding arithmetic), so the
// result is bitwise the same as without the tail (one-sweep Gauss-Seidel levels and every
// Kaczmarz form).
#include <cuda_runtime.h>

#include <algorithm>

#include "hz_common.cuh"
#include "hz_internal.h"
#include "hz_level.cuh"

namespace hz {

namespace {

constexpr int TAIL_THREADS = 1024;

template <class T>
__device__ __forceinline__ void tail_body(const TailArgs& A, const int* __restrict__ stop, const Inst& bi) {
  extern __shared__ __align__(16) unsigned char smem[];
  const c2<T>* fin = reinterpret_cast<const c2<T>*>(A.f_in) + blockIdx.z * bi.sf;
  c2<T>* uout = reinterpret_cast<c2<T>*>(A.u_out) + blockIdx.z * bi.so;
  auto U = [&](int l) { return reinterpret_cast<c2<T>*>(smem + A.lv[l].off_u); };
  auto F = [&](int l) { return reinterpret_cast<c2<T>*>(smem + A.lv[l].off_f); };
  auto K = [&](int l) { return reinterpret_cast<T*>(smem + A.lv[l].off_k); };
  auto D = [&](int l) { return reinterpret_cast<c2<T>*>(smem + A.lv[l].off_d); };
  auto V = [&](int l) { return reinterpret_cast<T*>(smem + A.lv[l].off_inv); };
  c2<T>* R = reinterpret_cast<c2<T>*>(smem + A.off_r);
  const int last = A.count - 1;

  // Kaczmarz levels are stored colour-blocked, the others row-major (lvl::Natural, lvl::Blocked)
  auto with_layout = [&](int l, auto&& fn) {
    const int nl = A.lv[l].n;
    if (A.lv[l].kind == TAIL_KACZ)
      fn(lvl::blocked(nl));
    else
      fn(lvl::Natural{nl + 1});
  };

  // Before the wait for the preceding kernel, everything that does not depend on it, so that with
  // programmatic dependent launch it overlaps that kernel: k H of every relaxation level (set up
  // once per problem), copied at once (cp.async, one wait) into K(l) on Gauss-Seidel levels and
  // into the cells of 1/|a|^2 on Kaczmarz levels, where the row constants replace it (plus a
  // row-major copy for the residual when there is room); the zero guess of the Kaczmarz levels.
  for (int l = 0; l < last; ++l) {
    const TailLevel& L = A.lv[l];
    const T* kh = reinterpret_cast<const T*>(L.kh);
    if (L.kind == TAIL_KACZ) {
      for (int q = threadIdx.x; q < lvl::blocked_cells(L.n); q += TAIL_THREADS) U(l)[q] = mk<T>(0, 0);
      T* kres = L.off_kres ? reinterpret_cast<T*>(smem + L.off_kres) : nullptr;
      lvl::for_nodes_blocked(L.n, [&](int q, int i, int j, int p) {
        const T* src = kh + (long long)j * L.pk + i;
        lvl::cp_async<sizeof(T)>(&V(l)[p], src);
        if (kres) lvl::cp_async<sizeof(T)>(&kres[q], src);
      });
    } else {
      const int w = L.n + 1;
      lvl::for_nodes(w, w * w, [&](int q, int i, int j) {
        lvl::cp_async<sizeof(T)>(&K(l)[q], kh + (long long)j * L.pk + i);
      });
    }
  }
  const int mc = (A.lv[last].n + 1) * (A.lv[last].n + 1);
  if (A.off_ainv) {  // the coarsest inverse, when it fits
    const c2<T>* src = reinterpret_cast<const c2<T>*>(A.ainvT);
    c2<T>* dst = reinterpret_cast<c2<T>*>(smem + A.off_ainv);
    for (int q = threadIdx.x; q < mc * mc; q += TAIL_THREADS) lvl::cp_async<sizeof(c2<T>)>(dst + q, src + q);
  }
  lvl::cp_async_wait_all();
  __syncthreads();
  for (int l = 0; l < last; ++l) {
    const TailLevel& L = A.lv[l];
    if (L.kind == TAIL_KACZ)
      lvl::for_blocked(L.n, [&](int i, int j, int p) {
        lvl::row_consts<T>(V(l)[p], i, j, L.n, (T)L.bA, &D(l)[p], &V(l)[p]);
      });
  }

  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;  // the whole block
  // the first level's right-hand side (the preceding kernel's output), and its red nodes if it is
  // a Gauss-Seidel level
  {
    const TailLevel& L = A.lv[0];
    const int w = L.n + 1;
    if (L.kind == TAIL_KACZ)
      lvl::for_nodes_blocked(L.n, [&](int, int i, int j, int p) {
        lvl::cp_async<sizeof(c2<T>)>(&F(0)[p], fin + (long long)j * A.pf + i);
      });
    else
      lvl::for_nodes(w, w * w, [&](int q, int i, int j) {
        lvl::cp_async<sizeof(c2<T>)>(&F(0)[q], fin + (long long)j * A.pf + i);
      });
    lvl::cp_async_wait_all();
    __syncthreads();
    if (L.kind == TAIL_GS) lvl::gs_red<T>(U(0), F(0), K(0), L.n, (T)L.bA);
  }
  __syncthreads();

  // down: relax from a zero guess (a Gauss-Seidel level's red nodes were set by the phase that
  // produced its right-hand side), residual with the (B) operator, full weighting
  for (int l = 0; l < last; ++l) {
    const TailLevel& L = A.lv[l];
    if (L.kind == TAIL_GS) {
      lvl::gs_black<T>(U(l), F(l), K(l), L.n, (T)L.bA);
      lvl::residual<T>(R, U(l), F(l), lvl::Natural{L.n + 1}, K(l), L.n + 1, L.n, (T)L.bB);
    } else {
      lvl::kacz_sweeps<T>(U(l), F(l), D(l), V(l), L.n, L.nu, false);
      if (L.off_kres)
        lvl::residual_blocked<T>(R, U(l), F(l), reinterpret_cast<const T*>(smem + L.off_kres), L.n + 1, L.n, (T)L.bB);
      else
        lvl::residual_blocked<T>(R, U(l), F(l), reinterpret_cast<const T*>(L.kh), L.pk, L.n, (T)L.bB);
    }
    __syncthreads();
    const TailLevel& C = A.lv[l + 1];
    if (C.kind == TAIL_GS)
      lvl::restrict_fw_red<T>(F(l + 1), U(l + 1), K(l + 1), (T)C.bA, R, L.n);
    else
      with_layout(l + 1, [&](auto lc) { lvl::restrict_fw<T>(F(l + 1), lc, R, L.n); });
    __syncthreads();
  }

  // coarsest: u = A^-1 f
  {
    const int m = (A.lv[last].n + 1) * (A.lv[last].n + 1);
    const c2<T>* ainvT = A.off_ainv ? reinterpret_cast<const c2<T>*>(smem + A.off_ainv)
                                    : reinterpret_cast<const c2<T>*>(A.ainvT);
    for (int r = threadIdx.x; r < m; r += TAIL_THREADS) U(last)[r] = lvl::coarse_row<T>(ainvT, F(last), m, r);
    __syncthreads();
  }

  // up: bilinear correction, relaxation in the reverse order (fused on Gauss-Seidel levels)
  for (int l = last - 1; l >= 0; --l) {
    const TailLevel& L = A.lv[l];
    if (L.kind == TAIL_GS) {
      with_layout(l + 1, [&](auto le) { lvl::gs_post_corrected<T>(U(l), F(l), K(l), L.n, (T)L.bA, U(l + 1), le); });
    } else {
      with_layout(l + 1, [&](auto le) { lvl::prolong_add<T>(U(l), lvl::blocked(L.n), U(l + 1), le, L.n); });
      __syncthreads();
      lvl::kacz_sweeps<T>(U(l), F(l), D(l), V(l), L.n, L.nu, true);
    }
  }

  const int w = A.lv[0].n + 1;
  if (A.lv[0].kind == TAIL_KACZ)
    lvl::for_nodes_blocked(A.lv[0].n, [&](int, int i, int j, int p) { uout[(long long)j * A.po + i] = U(0)[p]; });
  else
    lvl::for_nodes(w, w * w, [&](int q, int i, int j) { uout[(long long)j * A.po + i] = U(0)[q]; });
}

// The FP32 tail is held to 56 registers a thread, so that its 1024-thread block fits beside the
// deferred solution update (k_update_x, one 128-thread block per SM) that runs during the cycle.
__global__ void __maxnreg__(56) tail_kernel32(const TailArgs A, const int* __restrict__ stop, Inst bi) {
  tail_body<float>(A, stop, bi);
}
__global__ void __launch_bounds__(TAIL_THREADS) tail_kernel64(const TailArgs A, const int* __restrict__ stop, Inst bi) {
  tail_body<double>(A, stop, bi);
}

}  // namespace

size_t tail_layout(bool fp32, TailArgs* A) {
  const size_t c = fp32 ? sizeof(float2) : sizeof(double2), r = fp32 ? sizeof(float) : sizeof(double);
  size_t off = 0, rmax = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) & ~(size_t)15;
    return (unsigned)o;
  };
  for (int l = 0; l < A->count; ++l) {
    TailLevel& L = A->lv[l];
    const size_t Nn = (size_t)(L.n + 1) * (L.n + 1);
    const size_t N = L.kind == TAIL_KACZ ? (size_t)lvl::blocked_cells(L.n) : Nn;  // cells of u, f~, d, 1/|a|^2
    L.off_u = take(N * c);
    L.off_f = take(N * c);
    L.off_k = L.off_d = L.off_inv = 0;
    if (L.kind == TAIL_GS) L.off_k = take(N * r);
    if (L.kind == TAIL_KACZ) {
      L.off_d = take(N * c);
      L.off_inv = take(N * r);
    }
    if (L.kind != TAIL_COARSE) rmax = std::max(rmax, Nn);
  }
  for (int l = 0; l + 1 < A->count; ++l) {
    TailLevel& L = A->lv[l];
    const TailLevel& C = A->lv[l + 1];
    L.off_kres = 0;
    // the next level's u and f cells are contiguous; a Kaczmarz next level needs its zeroed u
    const size_t need = (size_t)(L.n + 1) * (L.n + 1) * r;
    const size_t nc = C.kind == TAIL_KACZ ? (size_t)lvl::blocked_cells(C.n) : (size_t)(C.n + 1) * (C.n + 1);
    if (L.kind == TAIL_KACZ && C.kind != TAIL_KACZ && need <= (size_t)(C.off_f - C.off_u) + nc * c) L.off_kres = C.off_u;
  }
  A->lv[A->count - 1].off_kres = 0;
  A->off_r = take(rmax * c);
  const size_t m = (size_t)(A->lv[A->count - 1].n + 1) * (A->lv[A->count - 1].n + 1);
  A->off_ainv = 0;
  if (off + m * m * c <= (size_t)TAIL_MAX_SMEM) A->off_ainv = take(m * m * c);
  return off;
}

cudaError_t launch_tail(bool fp32, const TailArgs& A, size_t smem, const int* stop, cudaStream_t s, const Inst& bi) {
  if (A.count < 2 || A.count > TAIL_MAX_LEVELS || smem > (size_t)TAIL_MAX_SMEM) return cudaErrorInvalidValue;
  static bool ready[2] = {false, false};
  cudaError_t e;
  if (!ready[fp32]) {
    e = fp32 ? cudaFuncSetAttribute(tail_kernel32, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_MAX_SMEM)
             : cudaFuncSetAttribute(tail_kernel64, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_MAX_SMEM);
    if (e) return e;
    ready[fp32] = true;
  }
  dim3 grid(1, 1, bi.count);
  if (fp32)
    pdl_launch(tail_kernel32, grid, TAIL_THREADS, smem, s, A, stop, bi);
  else
    pdl_launch(tail_kernel64, grid, TAIL_THREADS, smem, s, A, stop, bi);
  return cudaGetLastError();
}

}  // namespace hz
