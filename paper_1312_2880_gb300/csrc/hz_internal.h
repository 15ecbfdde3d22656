// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hz.h"

namespace hz {

// Launches `kernel` with programmatic stream serialization: it may begin launching while the
// previous kernel in the stream (or captured graph) is still running, and waits for it inside
// (every kernel of the library starts with pdl_enter()).
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Instances of one launch (multi right-hand-side batches): blockIdx.z selects the instance and
// every per-instance array advances by its stride in elements. su: the level's own arrays (u, u2,
// and f below the finest grid); sf: the right-hand side f; sc: the coarse level's arrays (fc,
// e_c); so: the output of the finest-grid post-sweep. The k h arrays and the coarsest inverse are
// shared. stop_stride: ints between the instances' stop flags.
struct Inst {
  int count = 1;
  long long su = 0, sf = 0, sc = 0, so = 0;
  int stop_stride = 0;
};

// ---------------------------------------------------------------- V-cycle kernel launchers
// `fp32` selects the working precision of the level arrays (float2/float instead of
// double2/double). `f64_src` says the right-hand side f is a double2 array even when fp32 is
// set (the finest level reads the FP64 Krylov vector directly). Pitches are in elements.
// `stop` is an optional device flag: when it is non-zero the kernel returns at once (used to
// turn the queued iterations after convergence into no-ops).

// omega != 1: red-black SOR (the relaxed value (1 - omega) u + omega u_GS).
cudaError_t launch_gs_colour(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh,
                             int pk, int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi = Inst(),
                             double omega = 1.0);
cudaError_t launch_gs_first(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh, int pk,
                            int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi = Inst(),
                            double omega = 1.0);
// One damped Jacobi sweep out of place (in == nullptr: from a zero guess).
cudaError_t launch_jacobi(bool fp32, void* out, int po, const void* in, int pu, const void* f, int pf, bool f64_src,
                          const void* kh, int pk, int n, double beta, double omega, const int* stop, cudaStream_t s,
                          const Inst& bi = Inst());
cudaError_t launch_kacz_colour(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh,
                               int pk, int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi = Inst());
cudaError_t launch_restrict_residual(bool fp32, void* fc, int pc, const void* u, int pu, const void* f, int pf,
                                     bool f64_src, const void* kh, int pk, int n, double beta, const int* stop,
                                     cudaStream_t s, const Inst& bi = Inst());
cudaError_t launch_prolong_add(bool fp32, void* u, int pu, const void* ec, int pc, int n, const int* stop,
                               cudaStream_t s, const Inst& bi = Inst());
cudaError_t launch_coarse_solve(bool fp32, void* u, int pu, const void* f, int pf, const void* ainvT, int nc,
                                const int* stop, cudaStream_t s, const Inst& bi = Inst());
// Fused passes for a Gauss-Seidel level with one sweep each way (hz_fused.cu). smooth_restrict
// writes u (pre-sweep from a zero guess) and fc (coarse right-hand side, h^2-scaled for the
// coarse level); prolong_smooth writes out = post-sweep(upre + P ec), as double2 when out_f64.
// variant: 0 = shared-memory tiles; 1 .. FUSED_VARIANTS-1 = register streaming (hz_stream.cu)
// with stream_rows(variant) rows per warp, in either form (inputs and outputs of the level's own
// precision).
constexpr int FUSED_VARIANTS = 9;
inline int stream_rows(int variant) { return 1 << variant; }
cudaError_t launch_smooth_restrict(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, bool f64_src,
                                   const void* kh, int pk, int n, double bA, double bB, const int* stop,
                                   cudaStream_t s, const Inst& bi = Inst(), int variant = 0);
cudaError_t launch_prolong_smooth(bool fp32, void* out, int po, bool out_f64, const void* upre, int pu, const void* ec,
                                  int pc, const void* f, int pf, bool f64_src, const void* kh, int pk, int n, double bA,
                                  const int* stop, cudaStream_t s, const Inst& bi = Inst(), int variant = 0);
// Register-streaming forms (FP32 or FP64; n >= 4; u / upre and kh rows 16-byte aligned).
cudaError_t launch_smooth_restrict_stream(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf,
                                          const void* kh, int pk, int n, double bA, double bB, int seg_rows,
                                          const int* stop, cudaStream_t s, const Inst& bi);
cudaError_t launch_prolong_smooth_stream(bool fp32, void* out, int po, const void* upre, int pu, const void* ec, int pc,
                                         const void* f, int pf, const void* kh, int pk, int n, double bA, int seg_rows,
                                         const int* stop, cudaStream_t s, const Inst& bi);
// Kaczmarz level kernels (hz_kaczmarz.cu). The whole-level pair keeps the level in one block's
// shared memory (at most KACZ_LEVEL_MAX_SMEM bytes: 28 or 56 bytes per node); the tile kernel runs
// one five-colour sweep per launch, out of place (uin may be null for a zero guess).
constexpr int KACZ_LEVEL_MAX_SMEM = 200 * 1024;
bool kacz_level_fits(bool fp32, int n);
cudaError_t launch_kacz_level_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                  int pk, int n, double bA, double bB, int nu, const int* stop, cudaStream_t s, const Inst& bi = Inst());
cudaError_t launch_kacz_level_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                   const void* kh, int pk, int n, double bA, int nu, const int* stop, cudaStream_t s, const Inst& bi = Inst());
// Whole level over a thread-block cluster (row bands, distributed shared memory; up to 16 blocks).
bool kacz_cluster_fits(bool fp32, int n);
cudaError_t launch_kacz_cluster_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                    int pk, int n, double bA, double bB, int nu, const int* stop, cudaStream_t s,
                                    const Inst& bi = Inst());
cudaError_t launch_kacz_cluster_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                     const void* kh, int pk, int n, double bA, int nu, const int* stop, cudaStream_t s,
                                     const Inst& bi = Inst());
// Whole level in global memory by one persistent cooperative launch per pass (hz_kgrid.cu); one
// instance (batch 1). Each block owns a band of grid rows and publishes its progress (phases
// done) in its counter; before a phase it waits, with a bounded number of polls, for the two
// neighbouring bands to have finished the previous one. The counters are zero at setup and all
// advance by the same amount in every launch of a level; err (shared by the levels) is set when a
// wait runs out and stays set until the host resets the region.
constexpr int KGRID_MAX_BLOCKS = 2048;
struct BandSync {
  unsigned int* err;
  unsigned int* ctr;  // KGRID_MAX_BLOCKS counters of one level
};
bool kacz_grid_available();  // cooperative launches supported, and capturable into a CUDA graph
cudaError_t launch_kacz_grid_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                 int pk, int n, double bA, double bB, int nu, const int* stop, BandSync bs,
                                 cudaStream_t s);
cudaError_t launch_kacz_grid_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                  const void* kh, int pk, int n, double bA, int nu, const int* stop, BandSync bs,
                                  cudaStream_t s);
// `sweeps` (1 or 2, from kacz_tile_sweeps_per_launch) Kaczmarz sweeps per launch over halo tiles.
int kacz_tile_sweeps_per_launch(bool fp32, int n, int nu);
cudaError_t launch_kacz_sweep_tile(bool fp32, void* uout, int po, const void* uin, int pu, const void* f, int pf,
                                   bool f64_src, const void* kh, int pk, int n, double bA, bool post, int sweeps,
                                   const int* stop, cudaStream_t s, const Inst& bi = Inst());
// Coarse tail (hz_tail.cu): levels lt .. L-1 of the V-cycle in one block's shared memory.
constexpr int TAIL_MAX_LEVELS = 12;
constexpr int TAIL_MAX_SMEM = 200 * 1024;
enum { TAIL_GS = 0, TAIL_KACZ = 1, TAIL_COARSE = 2 };
struct TailLevel {
  int n, kind, nu;   // n_l; TAIL_*; sweeps (Kaczmarz)
  double bA, bB;     // shift of the relaxation (A) and residual (B) operators
  const void* kh;    // k H of the level (device, working precision, pitch pk)
  int pk;
  unsigned off_u, off_f, off_k, off_d, off_inv;  // shared-memory byte offsets (tail_layout)
  // Kaczmarz levels: a row-major copy of k H for the residual, kept in the next level's u and f
  // cells (unused until the restriction writes them); 0: the residual reads k H from global memory
  unsigned off_kres;
};
struct TailArgs {
  int count;  // levels in the tail, the last the coarsest
  TailLevel lv[TAIL_MAX_LEVELS];
  unsigned off_r;    // residual scratch
  unsigned off_ainv; // coarsest inverse staged in shared memory when it fits (0: read from global)
  const void* ainvT; // coarsest inverse (transposed)
  const void* f_in;  // right-hand side of the first tail level (pitch pf)
  int pf;
  void* u_out;       // its final u (pitch po)
  int po;
};
// Fills the offsets; returns the shared memory the tail needs.
size_t tail_layout(bool fp32, TailArgs* A);
cudaError_t launch_tail(bool fp32, const TailArgs& A, size_t smem, const int* stop, cudaStream_t s,
                        const Inst& bi = Inst());
// dst (precision of fp32, pitch pd) = src (double2, pitch ps) * scale, on an (n+1)^2 grid.
cudaError_t launch_import(bool fp32, void* dst, int pd, const double2* src, int ps, int n, double scale,
                          cudaStream_t s);
// dst (double2, pitch pd) = src (precision of fp32, pitch ps) * scale.
cudaError_t launch_export(bool fp32, double2* dst, int pd, const void* src, int ps, int n, double scale,
                          const int* stop, cudaStream_t s);
cudaError_t launch_inject_kh(bool fp32, void* kh, int pk, const double* k0, int n0, int stride, int nl, double H,
                             cudaStream_t s);
// Dense inverse of the coarsest scaled operator, stored transposed in the working precision.
// work: 2 * m * m double2 scratch, m = (nc+1)^2. status: device int, 0 on success, 1 if singular.
cudaError_t launch_coarse_setup(bool fp32, void* ainvT, double2* work, const void* kh, int pk, int nc, double beta,
                                int* status, cudaStream_t s);

// ---------------------------------------------------------------- Krylov (FP64)

// Device-resident Bi-CGSTAB scalars and flags. Written by the last block of each reduction.
struct KState {
  double2 rho, rho_old, alpha, omega, beta, rv, ts;
  double bnorm2, tol2, ss, rr, tt, trr;
  int it;        // current iteration, 1-based
  int first;     // 1: the next direction update is p = r (start or restart)
  int done;      // 0 running, 1 recurrence converged, 2 breakdown, 3 non-finite, 4 maxit,
                 // 5 near-breakdown: renew the shadow residual at the next direction update
  int half;      // 1: converged after the half step (x += alpha y is then the step's only update)
  int hist_len;  // entries written to hist (may exceed hist_cap; extra entries are dropped)
  int hist_cap;
  int maxit;
  int iters_x2;  // twice the iteration count at the stop (half steps count .5)
  int shadow_restarts;  // near-breakdown restarts with a new shadow residual
  double rhat2;         // |r^|^2 of the current shadow residual
  double min_cos2;      // smallest |<r^, r>|^2 / (|r^|^2 |r|^2) seen in the solve (diagnostics)
  double min_step2;     // smallest |omega|^2 |t|^2 / |r|^2 seen while cos2 < stall_cos2 (diagnostics)
  double stall_cos2, stall_step2;  // near-breakdown thresholds of this solve (below)
  int max_shadow_restarts;
  // Deferred solution update (k_update_x): x += alpha_x y is due when xa is set (from k_apply_rv),
  // x += omega_x z when xw is set (from k_update_r); applied in that order.
  double2 alpha_x, omega_x;
  int xa, xw;
  unsigned int ticket[16];  // last-block counters, one per reduction kernel
};

enum { KT_INIT = 0, KT_RV, KT_S, KT_XA, KT_TS, KT_XR, KT_TRUE, KT_RESTART, KT_SHADOW, KT_XW };

// Shadow residual r^ (a reading of the paper's Bi-CGSTAB: pseudo-random instead of r^ = b).
constexpr unsigned long long SHADOW_SEED = 0x5EED1312ull;
// Near-breakdown (stalled recurrences): after an iteration with both
//   |<r^, r>|^2 < STALL_COS2 |r^|^2 |r|^2   and   |omega|^2 |t|^2 < STALL_STEP2 |r|^2
// the shadow residual is renewed (at most MAX_SHADOW_RESTARTS times per solve). Measured on the
// serving and parity workloads: converging solves keep the second ratio above 1.7e-5 whenever the
// first is below 1e-12; the two stalled ones reached 7.5e-20 and 5.2e-19. These are the defaults
// of hz_set_stall_detection.
constexpr double STALL_COS2 = 1e-12;
constexpr double STALL_STEP2 = 1e-8;
constexpr int MAX_SHADOW_RESTARTS = 16;

// Device-side loop of a solve graph (a WHILE conditional node): after every iteration the control
// kernel counts it and keeps the loop running while some instance of some problem is still
// iterating and the count is below the largest maxit + 2 (so the loop always ends).
constexpr int LOOP_MAX_PROBLEMS = 32;
struct LoopCtl {
  cudaGraphConditionalHandle handle;
  int* counter;  // device; zeroed by the graph before the loop
  int problems;
  KState* st[LOOP_MAX_PROBLEMS];  // each problem's KState array
  int batch[LOOP_MAX_PROBLEMS];
};
cudaError_t launch_loop_control(const LoopCtl& c, cudaStream_t s);

struct KrylovVecs {
  double2 *x, *r, *rhat, *p, *v, *s, *t, *y, *z, *tr;
  // FP32 V-cycle form: the preconditioner reads p32/s32 (p and s rounded to FP32 by the FP64
  // kernels that produce them) and writes y32 = K p, z32 = K s, which are computed in FP32 and
  // so held exactly in FP32; the FP64 kernels widen them in registers. Null in the FP64 form.
  float2 *p32, *s32, *y32, *z32;
  const double2* b;
  const double* kh;  // k h on the finest grid, pitch n+1
  int n;
  long long N;
  double scale_b;  // h^2: the solver works on the h^2-scaled system
  KState* st;        // [batch]
  double* partials;  // [batch][part_stride]
  double* hist;      // [batch][hist_stride]
  int G;             // reduction grid size
  // Batches of right-hand sides: instance b (blockIdx.z) uses every vector (b, x, r, p, v, s, t,
  // y, z, tr and the FP32 copies) advanced by b * sv elements, its own state, partials and
  // history; the shadow residual and k h are shared.
  int batch = 1;
  long long sv = 0;
  long long part_stride = 0;
  int hist_stride = 0;
  double stall_cos2 = STALL_COS2, stall_step2 = STALL_STEP2;  // copied into each KState at the start
  int max_shadow_restarts = MAX_SHADOW_RESTARTS;
};

// The vectors and state of instance b (host side, for launches that touch a single instance).
KrylovVecs instance_of(const KrylovVecs& k, int b);

cudaError_t launch_k_init(const KrylovVecs& k, double tol, int maxit, int hist_cap, cudaStream_t s);
cudaError_t launch_k_update_p(const KrylovVecs& k, cudaStream_t s);
cudaError_t launch_k_apply_rv(const KrylovVecs& k, cudaStream_t s);
cudaError_t launch_k_update_s(const KrylovVecs& k, cudaStream_t s);
cudaError_t launch_k_apply_ts(const KrylovVecs& k, cudaStream_t s);
cudaError_t launch_k_update_r(const KrylovVecs& k, cudaStream_t s);
// Half A (x += alpha y, omega_half false) or W (x += omega z) of the deferred solution update.
cudaError_t launch_k_update_x(const KrylovVecs& k, bool omega_half, cudaStream_t s);
cudaError_t launch_k_true_residual(const KrylovVecs& k, cudaStream_t s);
cudaError_t launch_k_restart(const KrylovVecs& k, cudaStream_t s);  // every instance of k (use instance_of for one)
// v = A u (scaled by out_scale) on the finest grid in FP64; beta = 0 for L, the shift for M.
cudaError_t launch_apply_fp64(double2* v, const double2* u, const double* kh, int n, double beta, double out_scale,
                              cudaStream_t s);

// ---------------------------------------------------------------- ray correction (hz_ray.cu)

// The Galerkin ray operator P^H A P in block-tridiagonal form and its block LU (hz_ray.cu): Nr
// rows of ray nodes, Bs = 8 Nr unknowns per block row; every block array holds Nr row-major
// Bs x Bs blocks (L[0] and U[Nr-1] unused), every vector Nr * Bs entries.
struct RayBlocks {
  int n = 0, m = 0, Nr = 0, Bs = 0;
  double2 *L = nullptr, *D = nullptr, *U = nullptr;     // assembled blocks (kept)
  double2 *Sinv = nullptr, *G = nullptr, *W = nullptr;  // S_J^{-1}, L_J S_{J-1}^{-1}, S_J^{-1} U_J
  double2 *g = nullptr, *z = nullptr, *y = nullptr, *e = nullptr, *dz = nullptr;  // solve vectors
  double2* fcol = nullptr;  // Bs: pivot column of the current Gauss-Jordan step
  int* perm = nullptr;      // Bs: pivot rows of the current inversion
  int* status = nullptr;    // device int: set to 1 by a zero or non-finite pivot column
};
cudaError_t launch_ray_phases(double2* ph, int n, double k, cudaStream_t s);
cudaError_t launch_ray_assemble(const RayBlocks& B, const double2* ph, const double* kh, cudaStream_t s);
cudaError_t launch_ray_restrict(double2* g, const double2* r, const double2* ph, int n, int m, cudaStream_t s);
cudaError_t launch_ray_prolong_add(double2* x, const double2* z, const double2* ph, int n, int m, cudaStream_t s);
cudaError_t ray_factor(const RayBlocks& B, cudaStream_t s);
// z = (P^H A P)^{-1} g by block substitution and one refinement step (z aliases neither g nor B's vectors).
cudaError_t ray_coarse_solve(const RayBlocks& B, double2* z, const double2* g, cudaStream_t s);
// r = b - v (v null: r untouched) and *out = |r|^2 (|b|^2), through ray_reduction_blocks() partials.
cudaError_t launch_ray_residual_norm(double2* r, const double2* b, const double2* v, long long N, double* partials,
                                     double* out, cudaStream_t s);
cudaError_t launch_ray_axpy(double2* x, const double2* z, long long N, cudaStream_t s);
int ray_reduction_blocks();

}  // namespace hz
