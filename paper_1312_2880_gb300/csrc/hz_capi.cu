// C ABI (include/hz.h): problem set-up, the level hierarchy of Sec. 5, the V-cycle driver, the
// graph-replayed Bi-CGSTAB loop of Sec. 6, the ray correction and stand-alone cycle solver of
// Sec. 6 (Table 7), and the step entry points used by the tests.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hz_internal.h"

using namespace hz;

namespace {

constexpr int HIST_CAP = 32768;       // device history entries (two per iteration)
constexpr int MAX_COARSE_UNKNOWNS = 1089;
constexpr int PARTIAL_SLOTS = 4;
constexpr int MAX_G = 16384;

// Scale bins in c = k_ref H: geometric midpoints between the paper's scales 0.3125, 0.625, 1.25
// and 2.5 (Sec. 4-5), and the guard band 1 < kH < 2 sqrt 2 for L relaxation.
const double BIN_LO = 0.625 / std::sqrt(2.0);
const double BIN_MID = 0.625 * std::sqrt(2.0);
const double BIN_HI = 1.25 * std::sqrt(2.0);
const double GUARD_LO = 1.0;
const double GUARD_HI = 2.0 * std::sqrt(2.0);
const double KACZ_BAND_LO = 0.625 * std::sqrt(2.0);
const double KACZ_BAND_HI = 2.0 * std::sqrt(2.0);

constexpr int PIPELINE = 3;  // polled mode: iterations queued ahead of the convergence poll

struct Level {
  int n = 0, pitch = 0;
  double H = 0;
  int relax_op = HZ_OP_L, smoother = HZ_SMOOTH_GS, resid_op = HZ_OP_L, nu = 1;
  void* kh = nullptr;  // k H, real, working precision
  int pk = 0;
  void* u = nullptr;  // working precision complex
  void* f = nullptr;  // working precision complex (levels >= 1)
  void* u2 = nullptr; // result of the fused post-smoothing pass (levels >= 1)
  int var_down = 0, var_up = 0;  // fused-pass variants (picked by the tile autotuner)
  int kform = 0;                 // hz_kacz_form of a Kaczmarz level (set up by plan_kaczmarz)
  double omega = 1.0;            // relaxation factor of a Jacobi or SOR level
};

struct Plan {
  int levels = 0;
  bool fp32 = false;
  std::vector<int> n, pitch;
  size_t total = 0;
  // offsets
  std::vector<size_t> off_kh, off_u, off_f, off_u2;
  size_t off_kh64 = 0, off_vec = 0, vec_bytes = 0, off_ainv = 0, off_work = 0, off_state = 0, off_partials = 0,
         off_hist = 0, off_status = 0, off_sync = 0, sync_bytes = 0;
  int nvec = 11;
  int m_coarse = 0;
  int batch = 1;
  std::vector<long long> ls;  // elements between instances of a level's arrays
  size_t rhat_bytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int auto_levels(int n) {
  int levels = 1, m = n;
  while (m % 2 == 0 && m > 8) {
    m /= 2;
    ++levels;
  }
  return levels;
}

bool make_plan(int n, const hz_hierarchy_opts& o, Plan* P, std::string* err) {
  int L = o.levels > 0 ? o.levels : auto_levels(n);
  if (L < 1 || L > 24) { *err = "levels out of range"; return false; }
  if (n % (1 << (L - 1)) != 0 || (n >> (L - 1)) < 2) {
    *err = "n is not divisible by 2^(levels-1) with at least 2 intervals on the coarsest grid";
    return false;
  }
  int nc = n >> (L - 1);
  if ((nc + 1) * (nc + 1) > MAX_COARSE_UNKNOWNS) {
    *err = "coarsest grid has more than 1089 unknowns; add levels";
    return false;
  }
  P->levels = L;
  P->fp32 = o.precision == HZ_PREC_FP32;
  const int B = o.batch < 1 ? 1 : o.batch;
  P->batch = B;
  P->ls.assign(L, 0);
  size_t ce = P->fp32 ? 8 : 16, re = P->fp32 ? 4 : 8;
  size_t off = 0;
  P->n.resize(L);
  P->pitch.resize(L);
  P->off_kh.assign(L, 0);
  P->off_u.assign(L, 0);
  P->off_f.assign(L, 0);
  P->off_u2.assign(L, 0);
  for (int l = 0; l < L; ++l) {
    int nl = n >> l;
    P->n[l] = nl;
    P->pitch[l] = ((nl + 1 + 31) / 32) * 32;
    size_t cells = (size_t)P->pitch[l] * (nl + 1);
    P->ls[l] = (long long)cells;
    if (l > 0 || P->fp32) {  // level 0 in FP64 reads the FP64 k h array directly
      P->off_kh[l] = off;
      off = align256(off + cells * re);
    }
    P->off_u[l] = off;
    off = align256(off + cells * ce * B);
    if (l > 0) {
      P->off_f[l] = off;
      off = align256(off + cells * ce * B);
      P->off_u2[l] = off;  // out-of-place result of the fused post-smoothing pass
      off = align256(off + cells * ce * B);
    } else if (o.gs_smoother == HZ_SMOOTH_JACOBI) {
      P->off_u2[0] = off;  // the other half of the finest level's Jacobi sweeps
      off = align256(off + cells * ce * B);
    }
  }
  size_t N = (size_t)(n + 1) * (n + 1);
  P->off_kh64 = off;
  off = align256(off + N * 8);
  P->vec_bytes = align256(N * 16 * B);  // one slot: B consecutive vectors
  P->rhat_bytes = P->vec_bytes;          // one shadow residual per instance (restarts renew it)
  P->off_vec = off;
  off += P->vec_bytes * (P->nvec - 1) + P->rhat_bytes;
  P->m_coarse = (nc + 1) * (nc + 1);
  P->off_ainv = off;
  off = align256(off + (size_t)P->m_coarse * P->m_coarse * ce);
  P->off_work = off;
  off = align256(off + (size_t)P->m_coarse * P->m_coarse * 2 * 16);
  P->off_state = off;
  off = align256(off + sizeof(KState) * B);
  P->off_partials = off;
  off = align256(off + (size_t)PARTIAL_SLOTS * MAX_G * 8 * B);
  P->off_hist = off;
  off = align256(off + (size_t)HIST_CAP * 8 * B);
  P->off_status = off;  // coarse-setup status, loop counter
  off = align256(off + 256);
  P->off_sync = off;  // error word and band counters of the grid-synchronised Kaczmarz form
  P->sync_bytes = align256(256 + (size_t)L * KGRID_MAX_BLOCKS * sizeof(unsigned int));
  off += P->sync_bytes;
  P->total = off;
  return true;
}

}  // namespace

struct hz_problem {
  int n = 0;
  double beta = 0.5;
  int bc = 0;
  std::vector<double> k_host;
  cudaStream_t user_stream = nullptr;  // the caller's stream (hz_set_stream)
  cudaStream_t stream = nullptr;       // the library's own non-blocking stream, fenced with user_stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  hz_hierarchy_opts opts{};
  bool setup = false;
  Plan plan;
  std::vector<Level> lv;
  unsigned char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  double* kh64 = nullptr;
  void* ainvT = nullptr;
  double2* work = nullptr;
  int* status_dev = nullptr;
  unsigned int* sync_dev = nullptr;  // grid-synchronised Kaczmarz form: error word, band counters
  KrylovVecs kv{};
  double2* b_int = nullptr;  // host-buffer solve: rhs and x on the device
  double2* x_int = nullptr;
  cudaGraphExec_t graph = nullptr;
  const double2* graph_b = nullptr;
  double2* graph_x = nullptr;
  int num_sms = 0;
  int* poll_host = nullptr;           // pinned: PIPELINE slots x batch x 4 ints (it, first, done, half)
  cudaEvent_t ev_poll[PIPELINE]{};    // completion of each polled iteration
  cudaGraphExec_t graph_iter = nullptr;  // one iteration, replayed from the host (polled mode)
  int tail_start = -1;  // first level run by the one-block coarse tail (-1: none)
  TailArgs tail{};
  size_t tail_smem = 0;
  std::string err;
  // Solve in flight (see solve_begin/solve_advance/solve_end).
  struct Run {
    enum Phase { IDLE = 0, RUNNING, POLLING, DONE };
    int phase = IDLE;
    double tol = 0;
    int maxit = 0;
    int restarts = 0;
    bool polled = false;       // host-polled iterations instead of the device-side loop
    long long launched = 0, seen = 0;
    double* user_x = nullptr;  // where solve_end copies the solution
  } run;
  KState* kstate_host = nullptr;  // pinned copy of the device Krylov state at the end of a solve
  cudaEvent_t ev_final = nullptr;
  // Side branch of an iteration: half of the deferred solution update (k_update_x) beside each
  // V-cycle, forked at its start and joined before its finest post-smoothing pass.
  cudaStream_t xstream = nullptr;
  cudaEvent_t ev_xfork = nullptr, ev_xjoin = nullptr;
  // Measurement: when set, every launch is followed by an event on `stream` (hz_profile_iteration).
  struct ProfRec { int kernel, level; cudaEvent_t ev; };
  std::vector<ProfRec>* prof = nullptr;
  bool prof_capture = false;  // prof events are recorded into a graph being captured
};

// Ray correction of one problem (hz_ray.cu): one device allocation holding the blocks, the
// solve vectors and the plane-wave table.
struct hz_ray {
  hz_problem* P = nullptr;
  double k = 0;
  RayBlocks B{};
  double2* ph = nullptr;  // 8 (n+1)^2: ph[j (n+1)^2 + p] = exp(i k d_j . x_p)
  void* mem = nullptr;
  bool own_mem = false;  // mem allocated by the library (no caller arena)
  size_t bytes = 0;
  double setup_ms = 0;
  // The ray solve B.z = (P^H A P)^{-1} B.g (about 4 (n/m + 1) chained launches) captured once.
  cudaGraphExec_t solve_graph = nullptr;
};

namespace {

// Orders the library stream after the caller's stream on entry and the caller's stream after the
// library stream on exit, so every call behaves as if issued on the caller's stream. (Graph
// capture is not allowed on the legacy default stream, so work never runs on it directly.)
struct StreamScope {
  hz_problem* P;
  explicit StreamScope(hz_problem* p) : P(p) {
    if (P && P->stream) {
      cudaEventRecord(P->ev_in, P->user_stream);
      cudaStreamWaitEvent(P->stream, P->ev_in, 0);
    }
  }
  ~StreamScope() {
    if (P && P->stream) {
      cudaEventRecord(P->ev_out, P->stream);
      cudaStreamWaitEvent(P->user_stream, P->ev_out, 0);
    }
  }
};

hz_status fail(hz_problem* p, hz_status st, const std::string& msg) {
  if (p) p->err = msg;
  return st;
}

hz_status cuda_fail(hz_problem* p, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(p, HZ_ECUDA, m);
}

#define CK(call)                                           \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return cuda_fail(P, e__, #call); \
  } while (0)

double op_beta(const hz_problem* P, int op) { return op == HZ_OP_M ? P->beta : 0.0; }

// Pass a launch's status through, recording a timing event after it when profiling.
cudaError_t mark(hz_problem* P, cudaError_t e, int kernel, int level) {
  if (e == cudaSuccess && P->prof) {
    cudaEvent_t ev;
    e = cudaEventCreate(&ev);
    // inside a stream capture the record becomes an event node of the graph
    if (e == cudaSuccess)
      e = P->prof_capture ? cudaEventRecordWithFlags(ev, P->stream, cudaEventRecordExternal)
                          : cudaEventRecord(ev, P->stream);
    if (e == cudaSuccess) P->prof->push_back({kernel, level, ev});
  }
  return e;
}

// Relaxation/residual roles of Sec. 5 for a non-coarsest level (the oracle's level_policy).
void level_roles(int variant, double c, const std::vector<double>& c_local, bool guard, int rule, Level* L) {
  // Kaczmarz levels (Sec. 4-5): with the band rule, every level with some node whose k(x) H lies
  // in [KACZ_BAND_LO, KACZ_BAND_HI), where red-black Gauss-Seidel is no smoother; with the bins
  // rule, the levels whose scale c = k_ref H is in the kH ~ 1.25 bin.
  bool kacz = false;
  if (rule == HZ_KACZ_RULE_BAND) {
    for (double v : c_local)
      if (v >= KACZ_BAND_LO && v < KACZ_BAND_HI) { kacz = true; break; }
  } else {
    kacz = (c >= BIN_MID && c < BIN_HI);
  }
  L->smoother = kacz ? HZ_SMOOTH_KACZMARZ : HZ_SMOOTH_GS;
  if (variant == HZ_VAR_SL_PLAIN) {
    L->relax_op = HZ_OP_M; L->smoother = HZ_SMOOTH_GS; L->resid_op = HZ_OP_M;
    return;
  }
  if (variant == HZ_VAR_SL) { L->relax_op = HZ_OP_M; L->resid_op = HZ_OP_M; return; }
  if (variant == HZ_VAR_HLM) { L->relax_op = HZ_OP_L; L->resid_op = HZ_OP_L; return; }
  L->resid_op = HZ_OP_L;
  L->relax_op = ((c >= BIN_LO && c < BIN_HI) || kacz) ? HZ_OP_M : HZ_OP_L;
  if (L->relax_op == HZ_OP_L && guard) {
    for (double v : c_local)
      if (v > GUARD_LO && v < GUARD_HI) { L->relax_op = HZ_OP_M; break; }
  }
}

// ------------------------------------------------------------------ V-cycle driver

struct Src {
  const void* f;
  int pf;
  bool f64;
};

const void* kh_of(const hz_problem* P, int l, int* pk) {
  if (l == 0 && !P->plan.fp32) { *pk = P->n + 1; return P->kh64; }
  *pk = P->lv[l].pk;
  return P->lv[l].kh;
}

// Launch instances: every right-hand side of the batch (solves) or instance 0 (step entry points).
Inst inst_for(const hz_problem* P, int l, bool all) {
  Inst bi;
  if (!all || P->plan.batch == 1) return bi;
  const Plan& pl = P->plan;
  bi.count = pl.batch;
  bi.su = pl.ls[l];
  bi.sf = l == 0 ? P->kv.sv : pl.ls[l];
  bi.sc = l + 1 < pl.levels ? pl.ls[l + 1] : 0;
  bi.so = l == 0 ? P->kv.sv : pl.ls[l];
  bi.stop_stride = (int)(sizeof(KState) / sizeof(int));
  return bi;
}

// A Gauss-Seidel level with one sweep each way runs as two fused tile passes (hz_fused.cu).
bool fused(const hz_problem* P, int l) {
  const Level& L = P->lv[l];
  return l < P->plan.levels - 1 && L.smoother == HZ_SMOOTH_GS && L.nu == 1;
}

// How a Kaczmarz level runs (hz_kacz_form): one launch per colour, the whole level in one block,
// one tiled launch per sweep (even sweep counts, ping-pong between u and u2 ending in u), or the
// whole level over a thread-block cluster. The finest level keeps the colour launches (its
// right-hand side is the FP64 Krylov vector in the FP32 form).
enum KaczPath { KACZ_COLOUR = HZ_KACZ_COLOUR, KACZ_LEVEL = HZ_KACZ_LEVEL, KACZ_TILE = HZ_KACZ_TILE,
                KACZ_CLUSTER = HZ_KACZ_CLUSTER, KACZ_GRID = HZ_KACZ_GRID };
// Band synchronisation of the grid-synchronised Kaczmarz form on level l (the problem's sync region:
// the error word, then KGRID_MAX_BLOCKS counters per level).
BandSync band_sync_of(const hz_problem* P, int l) {
  return BandSync{P->sync_dev, P->sync_dev + 64 + (size_t)l * KGRID_MAX_BLOCKS};
}
bool uses_grid_form(const hz_problem* P) {
  for (int l = 0; l + 1 < P->plan.levels; ++l)
    if (P->lv[l].smoother == HZ_SMOOTH_KACZMARZ && P->lv[l].kform == HZ_KACZ_GRID &&
        !(P->tail_start > 0 && l >= P->tail_start))
      return true;
  return false;
}
// After a synchronised solve: HZ_ETIMEOUT (and a reset barrier) if a grid barrier wait ran out.
hz_status grid_sync_check(hz_problem* P) {
  if (!uses_grid_form(P)) return HZ_OK;
  unsigned int err = 0;
  if (cudaMemcpy(&err, P->sync_dev, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess) return HZ_ECUDA;
  if (err == 0) return HZ_OK;
  cudaMemset(P->sync_dev, 0, P->plan.sync_bytes);  // counters back in step, error cleared
  return HZ_ETIMEOUT;
}

KaczPath kacz_path(const hz_problem* P, int l) {
  const Level& L = P->lv[l];
  if (L.smoother != HZ_SMOOTH_KACZMARZ) return KACZ_COLOUR;
  return (KaczPath)L.kform;
}
bool kform_ok(const hz_problem* P, int l, int form) {
  const Level& L = P->lv[l];
  const bool fp32 = P->plan.fp32;
  switch (form) {
    case HZ_KACZ_COLOUR: return true;
    case HZ_KACZ_LEVEL: return l > 0 && kacz_level_fits(fp32, L.n);
    case HZ_KACZ_TILE: return l > 0 && L.nu % 2 == 0;
    case HZ_KACZ_CLUSTER: return l > 0 && kacz_cluster_fits(fp32, L.n);
    case HZ_KACZ_GRID: return l > 0 && P->plan.batch == 1 && kacz_grid_available();
  }
  return false;
}
// Default form: FP32 - one block if the level fits, else a cluster, else tiles; FP64 - a cluster
// (the FP64 pipe of one SM bounds the one-block form), else tiles up to n_l = 512, else colour
// launches (the tiles' halo recomputation is FP64 work, which outweighs the saved launches on the
// largest levels). Measured per Bi-CGSTAB iteration (four level launches): FP32 n_l = 128 cluster
// 118 us, tiles 247 us; n_l = 256 cluster 240 us, tiles 259 us; FP64 n_l = 64 cluster 206 us,
// colour launches 820 us; FP64 in the n = 4096 solve's graph: n_l = 1024 tiles 2.67 ms, colour
// launches 2.39 ms; n_l = 512 0.94 and 1.21 ms; n_l = 256 0.58 and 0.92 ms. All forms give the
// same bits.
int default_kform(const hz_problem* P, int l) {
  // FP32 levels of n_l >= 256 with a multiple of 4 sweeps: two sweeps per tiled launch beat the
  // cluster (config 3, n_l = 256: 0.13 ms per iteration against 0.23)
  if (P->plan.fp32 && kacz_tile_sweeps_per_launch(true, P->lv[l].n, P->lv[l].nu) == 2 &&
      !kacz_level_fits(true, P->lv[l].n) && kform_ok(P, l, HZ_KACZ_TILE))
    return HZ_KACZ_TILE;
  const int order32[] = {HZ_KACZ_LEVEL, HZ_KACZ_CLUSTER, HZ_KACZ_TILE}, order64[] = {HZ_KACZ_CLUSTER, HZ_KACZ_TILE};
  const int* o = P->plan.fp32 ? order32 : order64;
  const int cnt = P->plan.fp32 ? 3 : (P->lv[l].n <= 512 ? 2 : 1);
  for (int q = 0; q < cnt; ++q)
    if (kform_ok(P, l, o[q])) return o[q];
  return HZ_KACZ_COLOUR;
}
void plan_kaczmarz(hz_problem* P) {
  for (int l = 0; l < P->plan.levels - 1; ++l) {
    Level& L = P->lv[l];
    L.kform = HZ_KACZ_COLOUR;
    if (L.smoother != HZ_SMOOTH_KACZMARZ) continue;
    const int want = P->opts.kacz_form;
    L.kform = (want >= 0 && kform_ok(P, l, want)) ? want : default_kform(P, l);
  }
}

// Tiled sweeps on level l: `first_in` is the input of the first sweep (null = zero guess). One or
// two sweeps per launch, ping-pong between u and u2 ending in u.
cudaError_t kacz_tile_sweeps(hz_problem* P, int l, Src f, const void* first_in, bool post, const int* stop,
                             const Inst& bi) {
  const Level& L = P->lv[l];
  int pk;
  const void* kh = kh_of(P, l, &pk);
  const void* in = first_in;
  const int per = kacz_tile_sweeps_per_launch(P->plan.fp32, L.n, L.nu), launches = L.nu / per;
  cudaError_t e;
  for (int k = 0; k < launches; ++k) {
    void* out = ((launches - 1 - k) % 2 == 0) ? L.u : L.u2;
    if ((e = mark(P, launch_kacz_sweep_tile(P->plan.fp32, out, L.pitch, in, L.pitch, f.f, f.pf, f.f64, kh, pk, L.n,
                                            op_beta(P, L.relax_op), post, per, stop, P->stream, bi),
                  HZ_K_KACZ_SWEEP, l)))
      return e;
    in = out;
  }
  return cudaSuccess;
}

// `sweeps` damped Jacobi sweeps on level l ending in lv[l].u, from a zero guess or from lv[l].u;
// ping-pong between u and u2 (from u with an odd count, u is first copied to u2).
cudaError_t jacobi_sweeps(hz_problem* P, int l, Src f, bool from_zero, int sweeps, const int* stop, const Inst& bi) {
  const Level& L = P->lv[l];
  const bool fp32 = P->plan.fp32;
  int pk;
  const void* kh = kh_of(P, l, &pk);
  cudaError_t e;
  const void* src = from_zero ? nullptr : L.u;
  if (!from_zero && sweeps % 2 == 1) {
    const size_t es = fp32 ? sizeof(float2) : sizeof(double2);
    if ((e = mark(P, cudaMemcpy2DAsync(L.u2, (size_t)L.pitch * es, L.u, (size_t)L.pitch * es, (size_t)(L.n + 1) * es,
                                       (L.n + 1) * bi.count, cudaMemcpyDeviceToDevice, P->stream),
                  HZ_K_JACOBI, l)))
      return e;
    src = L.u2;
  }
  for (int k = 0; k < sweeps; ++k) {
    void* dst = ((sweeps - 1 - k) % 2 == 0) ? L.u : L.u2;
    if ((e = mark(P, launch_jacobi(fp32, dst, L.pitch, src, L.pitch, f.f, f.pf, f.f64, kh, pk, L.n,
                                   op_beta(P, L.relax_op), L.omega, stop, P->stream, bi),
                  HZ_K_JACOBI, l)))
      return e;
    src = dst;
  }
  return cudaSuccess;
}

// Where level l's result after post-relaxation lives (what level l-1 interpolates).
void* final_u(const hz_problem* P, int l) {
  return (l > 0 && fused(P, l)) ? P->lv[l].u2 : P->lv[l].u;
}

// Pre-relaxation from a zero guess on level l into lv[l].u and the restricted residual into
// level l+1's f.
cudaError_t level_down(hz_problem* P, int l, Src f, const int* stop, bool all = false) {
  const Inst bi = inst_for(P, l, all);
  const Level& L = P->lv[l];
  const Level& C = P->lv[l + 1];
  bool fp32 = P->plan.fp32;
  int pk;
  const void* kh = kh_of(P, l, &pk);
  double bA = op_beta(P, L.relax_op), bB = op_beta(P, L.resid_op);
  cudaStream_t s = P->stream;
  void* u = L.u;
  int pu = L.pitch;
  cudaError_t e;
  if (fused(P, l))
    return mark(P, launch_smooth_restrict(fp32, u, pu, C.f, C.pitch, f.f, f.pf, f.f64, kh, pk, L.n, bA, bB, stop, s, bi,
                                          L.var_down),
                HZ_K_SMOOTH_RESTRICT, l);
  KaczPath kp = kacz_path(P, l);
  if (kp == KACZ_LEVEL)
    return mark(P, launch_kacz_level_pre(fp32, u, pu, C.f, C.pitch, f.f, f.pf, kh, pk, L.n, bA, bB, L.nu, stop, s, bi),
                HZ_K_KACZ_LEVEL, l);
  if (kp == KACZ_CLUSTER)
    return mark(P, launch_kacz_cluster_pre(fp32, u, pu, C.f, C.pitch, f.f, f.pf, kh, pk, L.n, bA, bB, L.nu, stop, s, bi),
                HZ_K_KACZ_CLUSTER, l);
  if (kp == KACZ_GRID)
    return mark(P, launch_kacz_grid_pre(fp32, u, pu, C.f, C.pitch, f.f, f.pf, kh, pk, L.n, bA, bB, L.nu, stop,
                                        band_sync_of(P, l), s),
                HZ_K_KACZ_GRID, l);
  if (kp == KACZ_TILE) {
    if ((e = kacz_tile_sweeps(P, l, f, nullptr, false, stop, bi))) return e;
    return mark(P, launch_restrict_residual(fp32, C.f, C.pitch, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, bB, stop, s, bi),
                HZ_K_RESTRICT, l);
  }
  if (L.smoother == HZ_SMOOTH_JACOBI) {
    if ((e = jacobi_sweeps(P, l, f, true, L.nu, stop, bi))) return e;
  } else if (L.smoother == HZ_SMOOTH_GS || L.smoother == HZ_SMOOTH_SOR) {
    const double w = L.omega;
    if ((e = mark(P, launch_gs_first(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, 0, bA, stop, s, bi, w), HZ_K_GS_FIRST, l))) return e;
    if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, 1, bA, stop, s, bi, w), HZ_K_GS_COLOUR, l))) return e;
    for (int it = 1; it < L.nu; ++it)
      for (int c = 0; c < 2; ++c)
        if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, c, bA, stop, s, bi, w), HZ_K_GS_COLOUR, l))) return e;
  } else {
    size_t ce = fp32 ? 8 : 16;
    if ((e = mark(P, cudaMemset2DAsync(u, (size_t)pu * ce, 0, (size_t)(L.n + 1) * ce, (L.n + 1) * bi.count, s),
                  HZ_K_ZERO, l)))
      return e;
    for (int it = 0; it < L.nu; ++it)
      for (int c = 0; c < 5; ++c)
        if ((e = mark(P, launch_kacz_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, c, bA, stop, s, bi), HZ_K_KACZ_COLOUR, l))) return e;
  }
  return mark(P, launch_restrict_residual(fp32, C.f, C.pitch, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, bB, stop, s, bi), HZ_K_RESTRICT, l);
}

// `sweeps` sweeps of the level's smoother on lv[l].u in place; post selects the ordering.
cudaError_t level_sweeps(hz_problem* P, int l, Src f, int sweeps, bool post, const int* stop, bool all = false) {
  const Inst bi = inst_for(P, l, all);
  const Level& L = P->lv[l];
  bool fp32 = P->plan.fp32;
  int pk;
  const void* kh = kh_of(P, l, &pk);
  double bA = op_beta(P, L.relax_op);
  cudaStream_t s = P->stream;
  void* u = L.u;
  int pu = L.pitch;
  cudaError_t e;
  if (L.smoother == HZ_SMOOTH_JACOBI) return jacobi_sweeps(P, l, f, false, sweeps, stop, bi);
  for (int it = 0; it < sweeps; ++it) {
    if (L.smoother == HZ_SMOOTH_GS || L.smoother == HZ_SMOOTH_SOR) {
      for (int q = 0; q < 2; ++q)
        if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, post ? 1 - q : q, bA, stop, s, bi,
                                          L.omega),
                      HZ_K_GS_COLOUR, l)))
          return e;
    } else {
      for (int q = 0; q < 5; ++q)
        if ((e = mark(P, launch_kacz_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, post ? 4 - q : q, bA, stop, s, bi),
                      HZ_K_KACZ_COLOUR, l)))
          return e;
    }
  }
  return cudaSuccess;
}

// Correction from level l+1 and post-relaxation of level l. The result goes to `out` (pitch po):
// on the finest level a double2 array, otherwise final_u(l).
cudaError_t level_up(hz_problem* P, int l, Src f, void* out, int po, const int* stop, bool all = false) {
  const Inst bi = inst_for(P, l, all);
  const Level& L = P->lv[l];
  const Level& C = P->lv[l + 1];
  bool fp32 = P->plan.fp32;
  const void* ec = final_u(P, l + 1);
  cudaError_t e;
  if (fused(P, l)) {
    int pk;
    const void* kh = kh_of(P, l, &pk);
    return mark(P, launch_prolong_smooth(fp32, out, po, false, L.u, L.pitch, ec, C.pitch, f.f, f.pf, f.f64, kh, pk,
                                         L.n, op_beta(P, L.relax_op), stop, P->stream, bi, L.var_up),
                HZ_K_PROLONG_SMOOTH, l);
  }
  KaczPath kp = kacz_path(P, l);
  if (kp == KACZ_LEVEL) {
    int pk;
    const void* kh = kh_of(P, l, &pk);
    return mark(P, launch_kacz_level_post(fp32, L.u, L.pitch, ec, C.pitch, f.f, f.pf, kh, pk, L.n,
                                          op_beta(P, L.relax_op), L.nu, stop, P->stream, bi),
                HZ_K_KACZ_LEVEL, l);
  }
  if (kp == KACZ_CLUSTER) {
    int pk;
    const void* kh = kh_of(P, l, &pk);
    return mark(P, launch_kacz_cluster_post(fp32, L.u, L.pitch, ec, C.pitch, f.f, f.pf, kh, pk, L.n,
                                            op_beta(P, L.relax_op), L.nu, stop, P->stream, bi),
                HZ_K_KACZ_CLUSTER, l);
  }
  if (kp == KACZ_GRID) {
    int pk;
    const void* kh = kh_of(P, l, &pk);
    return mark(P, launch_kacz_grid_post(fp32, L.u, L.pitch, ec, C.pitch, f.f, f.pf, kh, pk, L.n,
                                         op_beta(P, L.relax_op), L.nu, stop, band_sync_of(P, l), P->stream),
                HZ_K_KACZ_GRID, l);
  }
  if ((e = mark(P, launch_prolong_add(fp32, L.u, L.pitch, ec, C.pitch, L.n, stop, P->stream, bi), HZ_K_PROLONG, l))) return e;
  if (kp == KACZ_TILE) {
    if ((e = kacz_tile_sweeps(P, l, f, L.u, true, stop, bi))) return e;
  } else if ((e = level_sweeps(P, l, f, L.nu, true, stop, all))) {
    return e;
  }
  if (l == 0) {  // unfused finest level: copy its u to the output (same element type)
    size_t es = fp32 ? sizeof(float2) : sizeof(double2);
    return mark(P, cudaMemcpy2DAsync(out, (size_t)po * es, L.u, (size_t)L.pitch * es, (size_t)(L.n + 1) * es,
                                     (L.n + 1) * bi.count, cudaMemcpyDeviceToDevice, P->stream),
                HZ_K_EXPORT, 0);
  }
  return cudaSuccess;
}

cudaError_t coarse(hz_problem* P, const int* stop, bool all = false) {
  const Level& C = P->lv.back();
  const Inst bi = inst_for(P, P->plan.levels - 1, all);
  return mark(P, launch_coarse_solve(P->plan.fp32, C.u, C.pitch, C.f, C.pitch, P->ainvT, C.n, stop, P->stream, bi),
              HZ_K_COARSE, P->plan.levels - 1);
}

// Right-hand side of level l: the V-cycle input on the finest grid (double2 in the FP64 form,
// float2 in the FP32 form; pitch n+1), the level's own f below.
Src level_src(const hz_problem* P, int l, const void* f0) {
  return l == 0 ? Src{f0, P->n + 1, !P->plan.fp32} : Src{P->lv[l].f, P->lv[l].pitch, false};
}

// Half of the deferred solution update (omega_half: x += omega z, else x += alpha y) on the side
// stream; in line on the library stream in the FP64 form (whose V-cycle uses the FP64 pipe itself)
// and while every launch is being timed. *forked tells whether a join is due.
cudaError_t fork_x_update(hz_problem* P, bool omega_half, bool* forked) {
  *forked = false;
  if (P->prof || !P->plan.fp32) return mark(P, launch_k_update_x(P->kv, omega_half, P->stream), HZ_K_UPDATE_X, 0);
  cudaError_t e = cudaEventRecord(P->ev_xfork, P->stream);
  if (!e) e = cudaStreamWaitEvent(P->xstream, P->ev_xfork, 0);
  if (!e) e = launch_k_update_x(P->kv, omega_half, P->xstream);
  if (!e) e = cudaEventRecord(P->ev_xjoin, P->xstream);
  *forked = !e;
  return e;
}

// z = V-cycle(f0) with f0 already h^2-scaled; f0 and z (pitch n+1) are double2 in the FP64 form
// and float2 in the FP32 form. xhalf >= 0 runs that half of the deferred solution update beside
// the cycle (0: x += alpha y, 1: x += omega z), from after its finest pre-smoothing pass (which
// streams the finest grid through HBM at ~70% of the copy rate) until its finest post-smoothing
// pass, the only launch of the cycle that writes z.
cudaError_t run_vcycle(hz_problem* P, const void* f0, void* z, const int* stop, bool all = false, int xhalf = -1) {
  const int L = P->plan.levels, lt = P->tail_start;
  cudaError_t e;
  bool forked = false;
  const int down_end = lt > 0 ? lt : L - 1;
  for (int l = 0; l < down_end; ++l) {
    if ((e = level_down(P, l, level_src(P, l, f0), stop, all))) return e;
    if (l == 0 && xhalf >= 0 && (e = fork_x_update(P, xhalf == 1, &forked))) return e;
  }
  if (lt > 0) {
    const Inst bi = inst_for(P, lt, all);
    if ((e = mark(P, launch_tail(P->plan.fp32, P->tail, P->tail_smem, stop, P->stream, bi), HZ_K_TAIL, lt))) return e;
  } else if ((e = coarse(P, stop, all))) {
    return e;
  }
  for (int l = down_end - 1; l >= 0; --l) {
    if (l == 0 && forked && (e = cudaStreamWaitEvent(P->stream, P->ev_xjoin, 0))) return e;
    void* out = l == 0 ? (void*)z : final_u(P, l);
    int po = l == 0 ? P->n + 1 : P->lv[l].pitch;
    if ((e = level_up(P, l, level_src(P, l, f0), out, po, stop, all))) return e;
  }
  return cudaSuccess;
}

// One Bi-CGSTAB iteration (two preconditioner applications, Sec. 6). The solution update is
// deferred: x += alpha y of the previous step beside the first V-cycle, x += omega z beside the
// second (KState::xa, xw; k_update_x).
cudaError_t enqueue_iteration(hz_problem* P) {
  const KrylovVecs& k = P->kv;
  cudaStream_t s = P->stream;
  const int* stop = &k.st->done;
  cudaError_t e;
  const bool fp32 = P->plan.fp32;
  if ((e = mark(P, launch_k_update_p(k, s), HZ_K_UPDATE_P, 0))) return e;
  if ((e = run_vcycle(P, fp32 ? (const void*)k.p32 : k.p, fp32 ? (void*)k.y32 : k.y, stop, true, 0))) return e;
  if ((e = mark(P, launch_k_apply_rv(k, s), HZ_K_APPLY_RV, 0))) return e;
  if ((e = mark(P, launch_k_update_s(k, s), HZ_K_UPDATE_S, 0))) return e;
  if ((e = run_vcycle(P, fp32 ? (const void*)k.s32 : k.s, fp32 ? (void*)k.z32 : k.z, stop, true, 1))) return e;
  if ((e = mark(P, launch_k_apply_ts(k, s), HZ_K_APPLY_TS, 0))) return e;
  return mark(P, launch_k_update_r(k, s), HZ_K_UPDATE_R, 0);
}

// The solve graph: the loop counter is zeroed, then a WHILE conditional node runs body() (one
// Bi-CGSTAB iteration of every problem) followed by the loop control kernel for as long as that
// kernel keeps the condition set. The whole iteration sequence of a solve is one graph launch.
template <class Body>
cudaError_t build_loop_graph(cudaStream_t s, LoopCtl ctl, Body body, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e) return e;
  cudaGraphNode_t mset = nullptr, cond = nullptr;
  cudaMemsetParams mp = {};
  mp.dst = ctl.counter;
  mp.value = 0;
  mp.elementSize = sizeof(int);
  mp.width = 1;
  mp.height = 1;
  mp.pitch = sizeof(int);
  e = cudaGraphAddMemsetNode(&mset, g, nullptr, 0, &mp);
  if (!e) e = cudaGraphConditionalHandleCreate(&ctl.handle, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = ctl.handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (!e) e = cudaGraphAddNode(&cond, g, &mset, nullptr, 1, &cp);
  if (!e) e = cudaStreamBeginCaptureToGraph(s, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
  if (!e) {
    cudaError_t eb = body();
    if (!eb) eb = launch_loop_control(ctl, s);
    cudaGraph_t captured = nullptr;  // the conditional node's own body graph
    e = cudaStreamEndCapture(s, &captured);
    if (eb) e = eb;
  }
  if (!e) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

int* loop_counter(hz_problem* P) { return P->status_dev + 16; }  // inside the 256-byte status block

hz_status build_graph(hz_problem* P) {
  if (P->graph) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  LoopCtl ctl{};
  ctl.counter = loop_counter(P);
  ctl.problems = 1;
  ctl.st[0] = P->kv.st;
  ctl.batch[0] = P->plan.batch;
  cudaError_t e = build_loop_graph(P->stream, ctl, [&]() { return enqueue_iteration(P); }, &P->graph);
  if (e) return cuda_fail(P, e, "building the solve graph");
  P->graph_b = P->kv.b;
  P->graph_x = P->kv.x;
  return HZ_OK;
}

// One Bi-CGSTAB iteration as a plain graph, replayed from the host (polled mode).
hz_status build_iter_graph(hz_problem* P) {
  if (P->graph_iter) return HZ_OK;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_iteration(P);
  cudaError_t e2 = cudaStreamEndCapture(P->stream, &g);
  if (e) return cuda_fail(P, e, "capture of one Bi-CGSTAB iteration");
  if (e2) return cuda_fail(P, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&P->graph_iter, g, 0);
  cudaGraphDestroy(g);
  if (e) return cuda_fail(P, e, "cudaGraphInstantiate");
  return HZ_OK;
}

// Polled mode: one iteration graph, then the 16-byte flag block (it, first, done, half) of every
// instance into pinned memory, then an event the host polls.
cudaError_t enqueue_replay(hz_problem* P) {
  hz_problem::Run& R = P->run;
  cudaStream_t s = P->stream;
  cudaError_t e = cudaGraphLaunch(P->graph_iter, s);
  const int slot = (int)(R.launched % PIPELINE), B = P->plan.batch;
  if (!e)
    e = cudaMemcpy2DAsync(P->poll_host + 4 * B * slot, 4 * sizeof(int), &P->kv.st->it, sizeof(KState), 4 * sizeof(int),
                          B, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaEventRecord(P->ev_poll[slot], s);
  if (!e) ++R.launched;
  return e;
}

// ------------------------------------------------------------------ resumable solve
// A solve is a small state machine so that one host thread can drive many problems at once
// (hz_solve_start / hz_solve_poll / hz_solve_finish); hz_solve runs the same machine blocking.
// Two ways to run the iterations:
//  * device loop (blocking solves): the solve graph runs every iteration in one launch;
//  * polled (non-blocking solves): the host keeps PIPELINE iteration-graph launches in flight and
//    reads each one's flag copy when its event completes. Graphs with a device-side loop launched
//    on different streams were measured to run one after another, while plain graph launches
//    overlap, so concurrent solves (serving) use this mode.
// RUNNING: the iterations, the true residual and a copy of every instance's Krylov state are in
// flight behind ev_final; when they land, an instance whose recurrence converged but whose true
// residual did not is restarted from it (at most 8 times); otherwise the solve is DONE.

cudaError_t launch_final(hz_problem* P) {
  cudaStream_t s = P->stream;
  cudaError_t e = launch_k_update_x(P->kv, false, s);  // the last steps' pending solution update
  if (!e) e = launch_k_update_x(P->kv, true, s);
  if (!e) e = launch_k_true_residual(P->kv, s);
  if (!e) e = cudaMemcpyAsync(P->kstate_host, P->kv.st, sizeof(KState) * P->plan.batch, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaEventRecord(P->ev_final, s);
  return e;
}

// Start (or, after a restart, resume) the iterations in the run's mode.
cudaError_t launch_iterations(hz_problem* P) {
  hz_problem::Run& R = P->run;
  if (!R.polled) {
    cudaError_t e = cudaGraphLaunch(P->graph, P->stream);
    if (!e) e = launch_final(P);
    R.phase = hz_problem::Run::RUNNING;
    return e;
  }
  R.launched = R.seen = 0;
  R.phase = hz_problem::Run::POLLING;
  cudaError_t e = cudaSuccess;
  while (!e && R.launched < PIPELINE && R.launched < (long long)R.maxit + 2) e = enqueue_replay(P);
  return e;
}

hz_status solve_begin(hz_problem* P, const double* rhs, double* x, double tol, int maxit, bool polled = false) {
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (P->run.phase != hz_problem::Run::IDLE) return fail(P, HZ_EINVAL, "a solve is already in flight on this problem");
  if (!rhs || !x || !(tol > 0) || maxit < 1) return fail(P, HZ_EINVAL, "bad solve arguments");
  if ((const double*)rhs == x) return fail(P, HZ_EINVAL, "rhs and x may not alias");
  if (maxit > HIST_CAP / 2 - 1) maxit = HIST_CAP / 2 - 1;
  // The solve graph works on the problem's own rhs and x buffers, so it is built once per problem
  // (an instantiation per caller buffer would cost more than the two copies).
  const size_t bytes = sizeof(double2) * (size_t)P->kv.N * P->plan.batch;
  if ((const double2*)rhs != P->b_int)
    CK(cudaMemcpyAsync(P->b_int, rhs, bytes, cudaMemcpyDeviceToDevice, P->stream));
  P->kv.b = P->b_int;
  P->kv.x = P->x_int;
  if (polled) {
    hz_status st = build_iter_graph(P);
    if (st) return st;
  } else if (!P->graph || P->graph_b != P->kv.b || P->graph_x != P->kv.x) {
    hz_status st = build_graph(P);
    if (st) return st;
  }
  hz_problem::Run& R = P->run;
  R = hz_problem::Run();
  R.tol = tol;
  R.maxit = maxit;
  R.user_x = x;
  R.polled = polled;
  CK(launch_k_init(P->kv, tol, maxit, HIST_CAP, P->stream));
  CK(launch_iterations(P));
  return HZ_OK;
}

hz_status solve_advance(hz_problem* P, bool block, int* done) {
  hz_problem::Run& R = P->run;
  cudaStream_t s = P->stream;
  *done = 0;
  for (;;) {
    if (R.phase == hz_problem::Run::IDLE) return fail(P, HZ_EINVAL, "no solve in flight");
    if (R.phase == hz_problem::Run::DONE) {
      *done = 1;
      return HZ_OK;
    }
    if (R.phase == hz_problem::Run::POLLING) {
      const int slot = (int)(R.seen % PIPELINE);
      if (block) {
        CK(cudaEventSynchronize(P->ev_poll[slot]));
      } else {
        cudaError_t q = cudaEventQuery(P->ev_poll[slot]);
        if (q == cudaErrorNotReady) return HZ_OK;
        if (q != cudaSuccess) return cuda_fail(P, q, "cudaEventQuery");
      }
      const int B = P->plan.batch;
      const int* flags = P->poll_host + 4 * B * slot;
      ++R.seen;
      bool all_done = true;  // done 5 (shadow restart pending) is still iterating
      for (int b = 0; b < B; ++b) all_done = all_done && flags[4 * b + 2] != 0 && flags[4 * b + 2] != 5;
      const long long cap = (long long)R.maxit + 2;
      if (all_done || (R.seen >= R.launched && R.launched >= cap)) {
        CK(launch_final(P));
        R.phase = hz_problem::Run::RUNNING;
      } else if (R.launched < cap) {
        CK(enqueue_replay(P));
      }
      continue;
    }
    if (block) {
      CK(cudaEventSynchronize(P->ev_final));
    } else {
      cudaError_t q = cudaEventQuery(P->ev_final);
      if (q == cudaErrorNotReady) return HZ_OK;
      if (q != cudaSuccess) return cuda_fail(P, q, "cudaEventQuery");
    }
    bool restarted = false;
    if (R.restarts < 8) {
      for (int b = 0; b < P->plan.batch; ++b) {
        const KState& hs = P->kstate_host[b];
        if (hs.done == 1 && hs.bnorm2 > 0 && !(hs.trr <= hs.tol2) && hs.it < R.maxit) {
          CK(launch_k_restart(instance_of(P->kv, b), s));
          restarted = true;
        }
      }
    }
    if (restarted) {
      ++R.restarts;
      CK(launch_iterations(P));
      continue;
    }
    R.phase = hz_problem::Run::DONE;
  }
}

hz_status instance_status(const KState& hs, int maxit, double* iters) {
  *iters = hs.iters_x2 * 0.5;
  if (hs.done == 2) return HZ_EBREAKDOWN;
  if (hs.done == 3) return HZ_ENONFINITE;
  if (hs.done == 4 || hs.done == 0 || hs.done == 5) {
    *iters = (double)maxit;
    return HZ_EMAXIT;
  }
  // The recurrence converged but the true residual b - A x (the quantity that stops the solve)
  // did not follow, and the restarts from it are used up or maxit was reached.
  if (hs.bnorm2 > 0 && !(hs.trr <= hs.tol2)) return HZ_EMAXIT;
  return HZ_OK;
}

// Results of a finished solve: instance 0's history, `ninfo` infos (one per instance).
hz_status solve_end(hz_problem* P, double* history, int history_cap, hz_solve_info* info, int ninfo = 1) {
  hz_problem::Run& R = P->run;
  if (R.phase != hz_problem::Run::DONE) return fail(P, HZ_EINVAL, "the solve has not finished");
  R.phase = hz_problem::Run::IDLE;
  const int B = P->plan.batch;
  if (R.user_x && R.user_x != (double*)P->x_int)
    CK(cudaMemcpyAsync(R.user_x, P->x_int, sizeof(double2) * (size_t)P->kv.N * B, cudaMemcpyDeviceToDevice,
                       P->stream));
  double iters0 = 0;
  const hz_status st = instance_status(P->kstate_host[0], R.maxit, &iters0);
  int hl = std::min(P->kstate_host[0].hist_len, HIST_CAP);
  if (history && history_cap > 0 && hl > 0) {
    CK(cudaMemcpyAsync(history, P->kv.hist, sizeof(double) * std::min(hl, history_cap), cudaMemcpyDeviceToHost,
                       P->stream));
  }
  CK(cudaStreamSynchronize(P->stream));
  hz_status worst = HZ_OK;
  for (int b = 0; b < B; ++b) {
    const KState& hs = P->kstate_host[b];
    double it = 0;
    hz_status sb = instance_status(hs, R.maxit, &it);
    if (sb != HZ_OK && worst == HZ_OK) worst = sb;
    if (info && b < ninfo) {
      info[b].iterations = it;
      info[b].relres_true = hs.bnorm2 > 0 ? std::sqrt(hs.trr / hs.bnorm2) : 0.0;
      info[b].history_len = b == 0 ? std::min(hl, history_cap > 0 ? history_cap : 0) : 0;
      info[b].status = sb;
      info[b].restarts = R.restarts + hs.shadow_restarts;
    }
  }
  const hz_status res = B == 1 ? st : worst;
  const hz_status gsc = grid_sync_check(P);
  if (gsc == HZ_ETIMEOUT) return fail(P, gsc, "a grid-wide barrier wait of a Kaczmarz level ran out");
  if (gsc != HZ_OK) return fail(P, gsc, "reading the grid barrier state failed");
  if (res == HZ_EBREAKDOWN) return fail(P, res, "Bi-CGSTAB breakdown");
  if (res == HZ_ENONFINITE) return fail(P, res, "non-finite value in the Krylov scalars");
  if (res == HZ_EMAXIT) return fail(P, res, "maximum iterations reached");
  return HZ_OK;
}

hz_status solve_device(hz_problem* P, const double* rhs, double* x, double tol, int maxit, double* history,
                       int history_cap, hz_solve_info* info, int ninfo = 1) {
  hz_status st = solve_begin(P, rhs, x, tol, maxit);
  if (st) return st;
  int done = 0;
  st = solve_advance(P, true, &done);
  if (st) {
    P->run.phase = hz_problem::Run::IDLE;
    cudaStreamSynchronize(P->stream);
    return st;
  }
  return solve_end(P, history, history_cap, info, ninfo);
}

bool level_ok(const hz_problem* P, int level, bool allow_coarsest) {
  if (!P->setup) return false;
  if (level < 0 || level >= P->plan.levels) return false;
  if (!allow_coarsest && level == P->plan.levels - 1) return false;
  return true;
}

// Level-l right-hand side in working form (h^2-scaled) from a physical FP64 array.
cudaError_t import_rhs(hz_problem* P, int l, const double* f, Src* out) {
  double H = P->lv[l].H;
  if (l == 0 && P->plan.fp32) {
    *out = Src{P->kv.p32, P->n + 1, false};
    return launch_import(true, P->kv.p32, P->n + 1, (const double2*)f, P->n + 1, P->n, H * H, P->stream);
  }
  if (l == 0) {
    *out = Src{P->kv.tr, P->n + 1, true};
    return launch_import(false, P->kv.tr, P->n + 1, (const double2*)f, P->n + 1, P->n, H * H, P->stream);
  }
  *out = Src{P->lv[l].f, P->lv[l].pitch, false};
  return launch_import(P->plan.fp32, P->lv[l].f, P->lv[l].pitch, (const double2*)f, P->lv[l].n + 1, P->lv[l].n,
                       H * H, P->stream);
}

// Grids and per-level roles of the hierarchy (host only): the variant's rules of Sec. 5 with the
// scale c = k_ref H and the local values k(x) H by injection for the guard.
bool schedule(const hz_problem* P, const hz_hierarchy_opts& o, const Plan& pl, std::vector<Level>* out) {
  int n = P->n;
  double k_ref = o.k_ref;
  if (k_ref <= 0) {
    double sum = 0;
    for (double v : P->k_host) sum += v;
    k_ref = sum / P->k_host.size();
  }
  out->assign(pl.levels, Level());
  for (int l = 0; l < pl.levels; ++l) {
    Level& L = (*out)[l];
    L.n = pl.n[l];
    L.pitch = pl.pitch[l];
    L.H = 1.0 / L.n;
    L.pk = L.pitch;
    int stride = 1 << l;
    if (l == pl.levels - 1) {
      bool m_op = (o.variant == HZ_VAR_SL || o.variant == HZ_VAR_SL_PLAIN);
      L.relax_op = L.resid_op = m_op ? HZ_OP_M : HZ_OP_L;
      L.smoother = HZ_SMOOTH_DIRECT;
      L.nu = 0;
    } else {
      std::vector<double> c_local;
      c_local.reserve((size_t)(L.n + 1) * (L.n + 1));
      for (int j = 0; j <= L.n; ++j)
        for (int i = 0; i <= L.n; ++i)
          c_local.push_back(P->k_host[(size_t)stride * j * (n + 1) + (size_t)stride * i] * L.H);
      level_roles(o.variant, k_ref * L.H, c_local, o.guard != 0, o.kacz_rule, &L);
      L.nu = L.smoother == HZ_SMOOTH_KACZMARZ ? o.nu_kacz : o.nu_gs;
      if (L.smoother == HZ_SMOOTH_GS && o.gs_smoother != HZ_SMOOTH_GS) {
        L.smoother = o.gs_smoother;
        L.omega = o.omega > 0 ? o.omega : (o.gs_smoother == HZ_SMOOTH_JACOBI ? 0.8 : 1.0);
      }
    }
  }
  return true;
}

bool opts_ok(const hz_hierarchy_opts& o) {
  return !(o.variant < 0 || o.variant > 3 || (o.precision != 0 && o.precision != 1) || o.nu_gs < 1 || o.nu_gs > 8 ||
           o.nu_kacz < 1 || o.nu_kacz > 16 || o.k_ref < 0 || o.batch < 1 || o.batch > 1024 ||
           o.pass_variant < -1 || o.pass_variant >= FUSED_VARIANTS || o.coarse_tail < 0 || o.coarse_tail > 1 ||
           o.kacz_form < -1 || o.kacz_form > HZ_KACZ_GRID ||
           (o.gs_smoother != HZ_SMOOTH_GS && o.gs_smoother != HZ_SMOOTH_JACOBI && o.gs_smoother != HZ_SMOOTH_SOR) ||
           !(o.omega >= 0.0 && o.omega < 2.0) || (o.kacz_rule != HZ_KACZ_RULE_BAND && o.kacz_rule != HZ_KACZ_RULE_BINS));
}

// ------------------------------------------------------------------ coarse tail
// The largest tail that fits TAIL_MAX_SMEM: levels lt .. L-1 (lt >= 1), each a one-sweep
// Gauss-Seidel level or a Kaczmarz level, the last the coarsest.
void plan_tail(hz_problem* P) {
  P->tail_start = -1;
  const int L = P->plan.levels;
  if (!P->opts.coarse_tail || L < 3) return;
  const bool fp32 = P->plan.fp32;
  for (int lt = 1; lt <= L - 2; ++lt) {
    if (L - lt > TAIL_MAX_LEVELS) continue;
    bool ok = true;
    TailArgs A{};
    A.count = L - lt;
    for (int l = lt; l < L && ok; ++l) {
      const Level& V = P->lv[l];
      TailLevel& T = A.lv[l - lt];
      T.n = V.n;
      T.nu = V.nu;
      T.bA = op_beta(P, V.relax_op);
      T.bB = op_beta(P, V.resid_op);
      T.kh = V.kh;
      T.pk = V.pk;
      if (l == L - 1)
        T.kind = TAIL_COARSE;
      else if (fused(P, l))
        T.kind = TAIL_GS;
      else if (V.smoother == HZ_SMOOTH_KACZMARZ)
        T.kind = TAIL_KACZ;
      else
        ok = false;
    }
    if (!ok) continue;
    const size_t smem = tail_layout(fp32, &A);
    if (smem > (size_t)TAIL_MAX_SMEM) continue;
    A.ainvT = P->ainvT;
    A.f_in = P->lv[lt].f;
    A.pf = P->lv[lt].pitch;
    A.u_out = final_u(P, lt);
    A.po = P->lv[lt].pitch;
    P->tail = A;
    P->tail_smem = smem;
    P->tail_start = lt;
    return;
  }
}

// ------------------------------------------------------------------ tile autotuner
// Every fused Gauss-Seidel level runs each candidate variant of its two passes
// (shared-memory tiles, or register streaming with 2 .. 256 rows per warp) on its own arrays,
// with all right-hand sides of the batch: one untimed launch, then the best of three timings of
// five back-to-back launches with CUDA events on the library stream. The fastest is kept, and cached per
// (n_l, batch, pass, finest level or not, precision) for later problems of the same shape.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, int> g_tune_cache;

// Candidates for a level of n_l intervals: streaming needs n_l >= 4; segments longer than the
// level add nothing over the one that covers it.
std::vector<int> tune_candidates(int nl) {
  std::vector<int> c{0};
  if (nl < 4) return c;
  for (int v = 1; v < FUSED_VARIANTS; ++v) {
    c.push_back(v);
    if (stream_rows(v) >= nl + 1) break;
  }
  return c;
}

// Best of three timings of five back-to-back launches (after one untimed launch), in ms per launch.
cudaError_t time_pass(hz_problem* P, int l, bool up, float* best_ms) {
  cudaEvent_t a, b;
  cudaError_t e;
  if ((e = cudaEventCreate(&a))) return e;
  if ((e = cudaEventCreate(&b))) { cudaEventDestroy(a); return e; }
  const void* f0 = P->plan.fp32 ? (const void*)P->kv.p32 : (const void*)P->kv.p;
  void* out0 = P->plan.fp32 ? (void*)P->kv.y32 : (void*)P->kv.y;
  auto launch = [&]() -> cudaError_t {
    if (up) {
      void* out = l == 0 ? out0 : final_u(P, l);
      int po = l == 0 ? P->n + 1 : P->lv[l].pitch;
      return level_up(P, l, level_src(P, l, f0), out, po, nullptr, true);
    }
    return level_down(P, l, level_src(P, l, f0), nullptr, true);
  };
  constexpr int REPS = 5;
  *best_ms = 1e30f;
  e = launch();
  for (int rep = 0; rep < 3 && !e; ++rep) {
    e = cudaEventRecord(a, P->stream);
    for (int q = 0; q < REPS && !e; ++q) e = launch();
    if (!e) e = cudaEventRecord(b, P->stream);
    if (!e) e = cudaEventSynchronize(b);
    float ms = 0;
    if (!e) e = cudaEventElapsedTime(&ms, a, b);
    if (!e) *best_ms = std::min(*best_ms, ms / REPS);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

constexpr int FP64_TUNE_MIN_N = 2048;  // smallest FP64 level whose fused-pass form is tuned

cudaError_t autotune(hz_problem* P) {
  const int B = P->plan.batch;
  for (int l = 0; l < P->plan.levels - 1; ++l) {
    Level& L = P->lv[l];
    if (!fused(P, l) || (P->tail_start > 0 && l >= P->tail_start)) continue;  // tail levels run in hz_tail.cu
    if (P->opts.pass_variant >= 0) {
      const bool ok = P->opts.pass_variant == 0 || L.n >= 4;
      L.var_down = L.var_up = ok ? P->opts.pass_variant : 0;
      continue;
    }
    if (!P->plan.fp32 && L.n < FP64_TUNE_MIN_N) {
      // FP64 levels that fit L2 keep the tiles: the passes are bound by the FP64 pipe, the
      // streaming forms recompute halo rows (more FP64 work), and timed in the solve they were
      // slower at the finest level (n = 512: 80 us against 60 us per pre-pass), although
      // isolated launches ranked them ahead. Larger levels are tuned like FP32 ones (n = 4096,
      // per iteration in the solve's graph: pre-passes 4.79 ms with tiles, 3.82 ms with 32-row
      // streaming; post-passes 3.96 and 2.51 ms).
      L.var_down = L.var_up = 0;
      continue;
    }
    for (int up = 0; up < 2; ++up) {
      int& var = up ? L.var_up : L.var_down;
      const auto key = std::make_tuple(L.n, B, up, l == 0 ? 1 : 0, P->plan.fp32 ? 1 : 0);
      {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
          var = it->second;
          continue;
        }
      }
      int best = 0;
      float best_ms = 1e30f;
      std::vector<std::pair<int, float>> timed;
      for (int v : tune_candidates(L.n)) {
        var = v;
        float ms;
        cudaError_t e = time_pass(P, l, up, &ms);
        if (e) return e;
        timed.emplace_back(v, ms);
        if (ms < best_ms) { best_ms = ms; best = v; }
      }
      // Streaming forms within 5% of the fastest count as ties, and the tie goes to the longest
      // segment: isolated launches rank near-equal forms by noise, while in the solve's graph the
      // shorter segments were the slower ones (n = 512 wedge, finest post-pass: 4 rows per warp
      // instead of 8 cost 1.9 ms per solve).
      for (const auto& t : timed)
        if (best > 0 && t.first > best && t.second <= 1.05f * best_ms) best = t.first;
      var = best;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[key] = best;
    }
  }
  return cudaSuccess;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

void hz_default_opts(hz_hierarchy_opts* o) {
  if (!o) return;
  o->levels = 0;
  o->variant = HZ_VAR_HYB;
  o->precision = HZ_PREC_FP64;
  o->nu_gs = 1;
  o->nu_kacz = 4;
  o->guard = 1;
  o->k_ref = 0.0;
  o->batch = 1;
  o->pass_variant = -1;
  o->coarse_tail = 1;
  o->kacz_form = -1;
  o->gs_smoother = HZ_SMOOTH_GS;
  o->omega = 0.0;
  o->kacz_rule = HZ_KACZ_RULE_BAND;
}

hz_status hz_create_problem(int n, const double* k_field, double beta, int bc, hz_problem** out) {
  if (!out) return HZ_EINVAL;
  *out = nullptr;
  if (n < 2 || n > 32768 || !k_field || bc != HZ_BC_SOMMERFELD1 || !std::isfinite(beta) || beta < 0) return HZ_EINVAL;
  size_t N = (size_t)(n + 1) * (n + 1);
  for (size_t q = 0; q < N; ++q)
    if (!(k_field[q] > 0) || !std::isfinite(k_field[q])) return HZ_EINVAL;
  hz_problem* P = new hz_problem();
  P->n = n;
  P->beta = beta;
  P->bc = bc;
  P->k_host.assign(k_field, k_field + N);
  hz_default_opts(&P->opts);
  *out = P;
  return HZ_OK;
}

hz_status hz_set_stream(hz_problem* P, void* stream) {
  if (!P) return HZ_EINVAL;
  P->user_stream = (cudaStream_t)stream;
  return HZ_OK;
}

size_t hz_footprint_bytes(int n, const hz_hierarchy_opts* opts) {
  hz_hierarchy_opts o;
  if (opts) o = *opts; else hz_default_opts(&o);
  Plan pl;
  std::string err;
  if (n < 2 || !make_plan(n, o, &pl, &err)) return 0;
  return pl.total;
}

static void release(hz_problem* P) {
  if (P->graph) { cudaGraphExecDestroy(P->graph); P->graph = nullptr; }
  if (P->ev_in) { cudaEventDestroy(P->ev_in); P->ev_in = nullptr; }
  if (P->ev_final) { cudaEventDestroy(P->ev_final); P->ev_final = nullptr; }
  for (auto& e : P->ev_poll) if (e) { cudaEventDestroy(e); e = nullptr; }
  if (P->poll_host) { cudaFreeHost(P->poll_host); P->poll_host = nullptr; }
  if (P->graph_iter) { cudaGraphExecDestroy(P->graph_iter); P->graph_iter = nullptr; }
  if (P->kstate_host) { cudaFreeHost(P->kstate_host); P->kstate_host = nullptr; }
  P->run = hz_problem::Run();
  if (P->ev_out) { cudaEventDestroy(P->ev_out); P->ev_out = nullptr; }
  if (P->stream) { cudaStreamSynchronize(P->stream); cudaStreamDestroy(P->stream); P->stream = nullptr; }
  if (P->xstream) { cudaStreamSynchronize(P->xstream); cudaStreamDestroy(P->xstream); P->xstream = nullptr; }
  if (P->ev_xfork) { cudaEventDestroy(P->ev_xfork); P->ev_xfork = nullptr; }
  if (P->ev_xjoin) { cudaEventDestroy(P->ev_xjoin); P->ev_xjoin = nullptr; }
  if (P->own_arena && P->arena) cudaFree(P->arena);
  P->arena = nullptr;
  P->own_arena = false;
  P->setup = false;
}

hz_status hz_setup_hierarchy(hz_problem* P, const hz_hierarchy_opts* opts, void* arena, size_t arena_bytes) {
  if (!P) return HZ_EINVAL;
  hz_hierarchy_opts o;
  if (opts) o = *opts; else hz_default_opts(&o);
  if (!opts_ok(o)) return fail(P, HZ_EINVAL, "bad hierarchy options");
  Plan pl;
  std::string err;
  if (!make_plan(P->n, o, &pl, &err)) return fail(P, HZ_EINVAL, err);
  if (pl.levels < 2) return fail(P, HZ_EINVAL, "at least two levels are needed");
  if (arena && arena_bytes < pl.total) return fail(P, HZ_ENOMEM, "arena smaller than hz_footprint_bytes");
  if (arena && ((uintptr_t)arena & 255)) return fail(P, HZ_EINVAL, "arena must be 256-byte aligned");
  release(P);
  P->opts = o;
  P->plan = pl;
  if (arena) {
    P->arena = (unsigned char*)arena;
    P->arena_bytes = arena_bytes;
  } else {
    void* a = nullptr;
    cudaError_t e = cudaMalloc(&a, pl.total);
    if (e) return fail(P, HZ_ENOMEM, std::string("cudaMalloc of the arena: ") + cudaGetErrorString(e));
    P->arena = (unsigned char*)a;
    P->arena_bytes = pl.total;
    P->own_arena = true;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&P->xstream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->ev_xfork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_xjoin, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_final, cudaEventDisableTiming));
  CK(cudaMallocHost(&P->kstate_host, sizeof(KState) * pl.batch));
  CK(cudaMallocHost(&P->poll_host, sizeof(int) * 4 * PIPELINE * pl.batch));
  for (auto& e : P->ev_poll) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  StreamScope scope(P);
  unsigned char* A = P->arena;
  int n = P->n;
  bool fp32 = pl.fp32;
  cudaStream_t s = P->stream;
  // FP64 k h on the finest grid: upload k, multiply by h in place.
  P->kh64 = (double*)(A + pl.off_kh64);
  CK(cudaMemcpyAsync(P->kh64, P->k_host.data(), sizeof(double) * P->k_host.size(), cudaMemcpyHostToDevice, s));
  CK(launch_inject_kh(false, P->kh64, n + 1, P->kh64, n, 1, n, 1.0 / n, s));
  // Levels: roles (host), k H by injection (device).
  if (!schedule(P, o, pl, &P->lv)) return fail(P, HZ_EINVAL, "bad hierarchy options");
  for (int l = 0; l < pl.levels; ++l) {
    Level& L = P->lv[l];
    L.kh = (l > 0 || fp32) ? (void*)(A + pl.off_kh[l]) : nullptr;
    L.u = A + pl.off_u[l];
    L.f = l > 0 ? (void*)(A + pl.off_f[l]) : nullptr;
    L.u2 = (l > 0 || pl.off_u2[0]) ? (void*)(A + pl.off_u2[l]) : nullptr;
    int stride = 1 << l;
    if (L.kh) CK(launch_inject_kh(fp32, L.kh, L.pk, P->kh64, n, stride, L.n, (double)stride, s));
  }
  // Krylov vectors and scratch.
  KrylovVecs& k = P->kv;
  unsigned char* vb = A + pl.off_vec;
  k.rhat = (double2*)vb;
  vb += pl.rhat_bytes;
  double2** slots[] = {&k.r, &k.p, &k.v, &k.s, &k.t, &k.y, &k.z, &k.tr, &P->b_int, &P->x_int};
  for (int q = 0; q < pl.nvec - 1; ++q) *slots[q] = (double2*)(vb + q * pl.vec_bytes);
  k.x = nullptr;
  k.b = nullptr;
  const long long Nn = (long long)(n + 1) * (n + 1);
  k.batch = pl.batch;
  k.sv = Nn;
  k.part_stride = (long long)PARTIAL_SLOTS * MAX_G;
  k.hist_stride = HIST_CAP;
  if (fp32) {  // FP32 copies packed into the y and z slots (16 bytes per node hold two float2 arrays)
    k.y32 = (float2*)k.y;
    k.p32 = k.y32 + Nn * pl.batch;
    k.z32 = (float2*)k.z;
    k.s32 = k.z32 + Nn * pl.batch;
  } else {
    k.p32 = k.s32 = k.y32 = k.z32 = nullptr;
  }
  k.kh = P->kh64;
  k.n = n;
  k.N = (long long)(n + 1) * (n + 1);
  k.scale_b = 1.0 / ((double)n * n);
  k.st = (KState*)(A + pl.off_state);
  k.partials = (double*)(A + pl.off_partials);
  k.hist = (double*)(A + pl.off_hist);
  // About four nodes per thread, between two and eight blocks per SM: on small grids fewer blocks
  // mean fewer block reductions (n = 512: 2 per SM), on large ones more warps hide the FP64 and
  // memory latency (n = 4096 update of x and r: 0.54 ms with 8 per SM, 0.60 ms with 2).
  long long want = (k.N + 4 * 256 - 1) / (4 * 256);
  want = std::max(want, std::min(2LL * P->num_sms, (k.N + 255) / 256));
  k.G = (int)std::min<long long>(want, std::min(8LL * P->num_sms, (long long)MAX_G));
  if (k.G < 1) k.G = 1;
  CK(cudaMemsetAsync(k.st, 0, sizeof(KState) * pl.batch, s));
  // Coarsest: dense inverse on the device.
  Level& C = P->lv.back();
  P->ainvT = A + pl.off_ainv;
  P->work = (double2*)(A + pl.off_work);
  P->status_dev = (int*)(A + pl.off_status);
  P->sync_dev = (unsigned int*)(A + pl.off_sync);
  CK(cudaMemsetAsync(P->sync_dev, 0, pl.sync_bytes, s));
  CK(launch_coarse_setup(fp32, P->ainvT, P->work, C.kh, C.pk, C.n, op_beta(P, C.relax_op), P->status_dev, s));
  int status = 1;
  CK(cudaMemcpyAsync(&status, P->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (status != 0) return fail(P, HZ_EINVAL, "coarsest operator is singular");
  plan_kaczmarz(P);
  plan_tail(P);
  CK(autotune(P));
  CK(cudaStreamSynchronize(s));
  P->setup = true;
  return HZ_OK;
}

int hz_describe_hierarchy(const hz_problem* P, const hz_hierarchy_opts* opts, hz_level_info* out, int cap) {
  if (!P || (cap > 0 && !out)) return -1;
  hz_hierarchy_opts o;
  if (opts) o = *opts; else hz_default_opts(&o);
  if (!opts_ok(o)) return -1;
  Plan pl;
  std::string err;
  if (!make_plan(P->n, o, &pl, &err) || pl.levels < 2) return -1;
  std::vector<Level> lv;
  schedule(P, o, pl, &lv);
  for (int l = 0; l < pl.levels && l < cap; ++l) {
    out[l].n = lv[l].n;
    out[l].H = lv[l].H;
    out[l].relax_op = lv[l].relax_op;
    out[l].smoother = lv[l].smoother;
    out[l].resid_op = lv[l].resid_op;
    out[l].nu = lv[l].nu;
    out[l].pass_down = out[l].pass_up = -1;  // chosen at setup
    out[l].in_tail = 0;
    out[l].kacz_form = -1;
  }
  return pl.levels;
}

int hz_num_levels(const hz_problem* P) { return (P && P->setup) ? P->plan.levels : 0; }

hz_status hz_get_level_info(const hz_problem* P, int level, hz_level_info* info) {
  if (!P || !info) return HZ_EINVAL;
  if (!P->setup) return HZ_ENOTSETUP;
  if (level < 0 || level >= P->plan.levels) return HZ_EINVAL;
  const Level& L = P->lv[level];
  info->n = L.n;
  info->H = L.H;
  info->relax_op = L.relax_op;
  info->smoother = L.smoother;
  info->resid_op = L.resid_op;
  info->nu = L.nu;
  const bool fz = level < P->plan.levels - 1 && fused(P, level) && !(P->tail_start > 0 && level >= P->tail_start);
  info->pass_down = fz ? L.var_down : -1;
  info->pass_up = fz ? L.var_up : -1;
  info->in_tail = (P->tail_start > 0 && level >= P->tail_start) ? 1 : 0;
  info->kacz_form = (L.smoother == HZ_SMOOTH_KACZMARZ && !info->in_tail) ? L.kform : -1;
  return HZ_OK;
}

static hz_status vcycle_dev(hz_problem* P, const double* r, double* z) {
  double h = 1.0 / P->n;
  if (P->plan.fp32) {
    CK(launch_import(true, P->kv.p32, P->n + 1, (const double2*)r, P->n + 1, P->n, h * h, P->stream));
    CK(run_vcycle(P, P->kv.p32, P->kv.y32, nullptr));
    CK(launch_export(true, (double2*)z, P->n + 1, P->kv.y32, P->n + 1, P->n, 1.0, nullptr, P->stream));
  } else {
    CK(launch_import(false, P->kv.p, P->n + 1, (const double2*)r, P->n + 1, P->n, h * h, P->stream));
    CK(run_vcycle(P, P->kv.p, z, nullptr));
  }
  return HZ_OK;
}

hz_status hz_vcycle(hz_problem* P, const double* r, double* z) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!r || !z || (const double*)r == z) return fail(P, HZ_EINVAL, "bad vcycle arguments");
  StreamScope scope(P);
  return vcycle_dev(P, r, z);
}

hz_status hz_solve_batch(hz_problem* P, const double* rhs, double* x, double tol, int maxit, hz_solve_info* infos) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  StreamScope scope(P);
  return solve_device(P, rhs, x, tol, maxit, nullptr, 0, infos, P->plan.batch);
}

hz_status hz_solve(hz_problem* P, const double* rhs, double* x, double tol, int maxit, double* history,
                   int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  if (P->setup && P->plan.batch != 1) return fail(P, HZ_EINVAL, "batched hierarchy: use hz_solve_batch");
  StreamScope scope(P);
  return solve_device(P, rhs, x, tol, maxit, history, history_cap, info);
}

hz_status hz_solve_host(hz_problem* P, const double* rhs_host, double* x_host, double tol, int maxit,
                        double* history, int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!rhs_host || !x_host) return fail(P, HZ_EINVAL, "null host pointer");
  if (P->plan.batch != 1) return fail(P, HZ_EINVAL, "batched hierarchy: use hz_solve_batch");
  StreamScope scope(P);
  size_t bytes = sizeof(double2) * (size_t)(P->n + 1) * (P->n + 1);
  CK(cudaMemcpyAsync(P->b_int, rhs_host, bytes, cudaMemcpyHostToDevice, P->stream));
  hz_status st = solve_device(P, (const double*)P->b_int, (double*)P->x_int, tol, maxit, history, history_cap, info);
  if (st != HZ_OK && st != HZ_EMAXIT && st != HZ_EBREAKDOWN && st != HZ_ENONFINITE) return st;
  CK(cudaMemcpyAsync(x_host, P->x_int, bytes, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return st;
}

hz_status hz_solve_start(hz_problem* P, const double* rhs, double* x, double tol, int maxit) {
  if (!P) return HZ_EINVAL;
  if (P->setup && P->plan.batch != 1) return fail(P, HZ_EINVAL, "batched hierarchy: use hz_solve_batch");
  StreamScope scope(P);
  return solve_begin(P, rhs, x, tol, maxit, true);
}

hz_status hz_solve_poll(hz_problem* P, int* done) {
  if (!P || !done) return HZ_EINVAL;
  hz_status st = solve_advance(P, false, done);
  if (st && st != HZ_EINVAL) {
    P->run.phase = hz_problem::Run::IDLE;
    cudaStreamSynchronize(P->stream);
  }
  return st;
}

hz_status hz_solve_finish(hz_problem* P, double* history, int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  StreamScope scope(P);
  int done = 0;
  hz_status st = solve_advance(P, true, &done);
  if (st) {
    P->run.phase = hz_problem::Run::IDLE;
    cudaStreamSynchronize(P->stream);
    return st;
  }
  return solve_end(P, history, history_cap, info);
}

hz_status hz_apply(hz_problem* P, int op, const double* u, double* v) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!u || !v || (const double*)u == v || (op != HZ_OP_L && op != HZ_OP_M)) return fail(P, HZ_EINVAL, "bad apply arguments");
  StreamScope scope(P);
  double n2 = (double)P->n * P->n;
  CK(launch_apply_fp64((double2*)v, (const double2*)u, P->kh64, P->n, op_beta(P, op), n2, P->stream));
  return HZ_OK;
}

hz_status hz_level_presmooth(hz_problem* P, int level, const double* f, double* u, double* fc) {
  if (!P) return HZ_EINVAL;
  if (!level_ok(P, level, false) || !f || !u || !fc) return fail(P, HZ_EINVAL, "bad level or pointer");
  StreamScope scope(P);
  Src src;
  CK(import_rhs(P, level, f, &src));
  CK(level_down(P, level, src, nullptr));
  const Level& L = P->lv[level];
  const Level& C = P->lv[level + 1];
  CK(launch_export(P->plan.fp32, (double2*)u, L.n + 1, L.u, L.pitch, L.n, 1.0, nullptr, P->stream));
  CK(launch_export(P->plan.fp32, (double2*)fc, C.n + 1, C.f, C.pitch, C.n, 1.0 / (C.H * C.H), nullptr, P->stream));
  return HZ_OK;
}

hz_status hz_level_postsmooth(hz_problem* P, int level, const double* f, const double* u_pre, const double* ec,
                              double* u) {
  if (!P) return HZ_EINVAL;
  if (!level_ok(P, level, false) || !f || !u_pre || !ec || !u) return fail(P, HZ_EINVAL, "bad level or pointer");
  StreamScope scope(P);
  Src src;
  CK(import_rhs(P, level, f, &src));
  const Level& L = P->lv[level];
  const Level& C = P->lv[level + 1];
  bool fp32 = P->plan.fp32;
  CK(launch_import(fp32, L.u, L.pitch, (const double2*)u_pre, L.n + 1, L.n, 1.0, P->stream));
  CK(launch_import(fp32, final_u(P, level + 1), C.pitch, (const double2*)ec, C.n + 1, C.n, 1.0, P->stream));
  if (level == 0 && fp32) {
    CK(level_up(P, 0, src, P->kv.y32, P->n + 1, nullptr));
    CK(launch_export(true, (double2*)u, P->n + 1, P->kv.y32, P->n + 1, P->n, 1.0, nullptr, P->stream));
  } else if (level == 0) {
    CK(level_up(P, 0, src, P->kv.v, P->n + 1, nullptr));
    CK(cudaMemcpyAsync(u, P->kv.v, sizeof(double2) * (size_t)(P->n + 1) * (P->n + 1), cudaMemcpyDeviceToDevice,
                       P->stream));
  } else {
    void* out = final_u(P, level);
    CK(level_up(P, level, src, out, L.pitch, nullptr));
    CK(launch_export(fp32, (double2*)u, L.n + 1, out, L.pitch, L.n, 1.0, nullptr, P->stream));
  }
  return HZ_OK;
}

hz_status hz_level_sweeps(hz_problem* P, int level, const double* f, double* u, int sweeps, int post) {
  if (!P) return HZ_EINVAL;
  if (!level_ok(P, level, false) || !f || !u || sweeps < 0) return fail(P, HZ_EINVAL, "bad level or pointer");
  StreamScope scope(P);
  Src src;
  CK(import_rhs(P, level, f, &src));
  const Level& L = P->lv[level];
  bool fp32 = P->plan.fp32;
  CK(launch_import(fp32, L.u, L.pitch, (const double2*)u, L.n + 1, L.n, 1.0, P->stream));
  CK(level_sweeps(P, level, src, sweeps, post != 0, nullptr));
  CK(launch_export(fp32, (double2*)u, L.n + 1, L.u, L.pitch, L.n, 1.0, nullptr, P->stream));
  return HZ_OK;
}

hz_status hz_coarse_solve(hz_problem* P, const double* f, double* u) {
  if (!P) return HZ_EINVAL;
  if (!P->setup || !f || !u) return fail(P, HZ_EINVAL, "bad arguments");
  int l = P->plan.levels - 1;
  const Level& C = P->lv[l];
  bool fp32 = P->plan.fp32;
  StreamScope scope(P);
  CK(launch_import(fp32, C.f, C.pitch, (const double2*)f, C.n + 1, C.n, C.H * C.H, P->stream));
  CK(coarse(P, nullptr));
  CK(launch_export(fp32, (double2*)u, C.n + 1, C.u, C.pitch, C.n, 1.0, nullptr, P->stream));
  return HZ_OK;
}

int hz_profile_iteration(hz_problem* P, const double* rhs, double* x, int iterations, hz_kernel_time* out, int cap) {
  if (!P || !P->setup || !rhs || !x || iterations < 1 || (cap > 0 && !out)) return -1;
  StreamScope scope(P);
  std::vector<hz_problem::ProfRec> recs;
  cudaEvent_t start;
  if (cudaEventCreate(&start) != cudaSuccess) return -1;
  P->kv.b = (const double2*)rhs;
  P->kv.x = (double2*)x;
  int count = -1;
  cudaError_t e = launch_k_init(P->kv, 1e-300, iterations + 1, HIST_CAP, P->stream);
  if (e == cudaSuccess) e = cudaEventRecord(start, P->stream);
  P->prof = &recs;
  for (int it = 0; it < iterations && e == cudaSuccess; ++it) e = enqueue_iteration(P);
  P->prof = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e == cudaSuccess) {
    cudaEvent_t prev = start;
    count = (int)recs.size();
    for (int q = 0; q < count; ++q) {
      float ms = 0;
      cudaEventElapsedTime(&ms, prev, recs[q].ev);
      if (q < cap) out[q] = hz_kernel_time{recs[q].kernel, recs[q].level, ms};
      prev = recs[q].ev;
    }
  } else {
    cuda_fail(P, e, "hz_profile_iteration");
  }
  for (auto& r : recs) cudaEventDestroy(r.ev);
  cudaEventDestroy(start);
  return count;
}

int hz_profile_graph(hz_problem* P, const double* rhs, double* x, int iterations, hz_kernel_time* out, int cap) {
  if (!P || !P->setup || !rhs || !x || iterations < 1 || (cap > 0 && !out)) return -1;
  StreamScope scope(P);
  std::vector<hz_problem::ProfRec> recs;
  cudaEvent_t start;
  if (cudaEventCreate(&start) != cudaSuccess) return -1;
  P->kv.b = (const double2*)rhs;
  P->kv.x = (double2*)x;
  int count = -1;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = launch_k_init(P->kv, 1e-300, iterations + 1, HIST_CAP, P->stream);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ec = cudaEventRecordWithFlags(start, P->stream, cudaEventRecordExternal);
    P->prof = &recs;
    P->prof_capture = true;
    for (int it = 0; it < iterations && ec == cudaSuccess; ++it) ec = enqueue_iteration(P);
    P->prof = nullptr;
    P->prof_capture = false;
    e = cudaStreamEndCapture(P->stream, &g);
    if (ec) e = ec;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e == cudaSuccess) {
    cudaEvent_t prev = start;
    count = (int)recs.size();
    for (int q = 0; q < count; ++q) {
      float ms = 0;
      cudaEventElapsedTime(&ms, prev, recs[q].ev);
      if (q < cap) out[q] = hz_kernel_time{recs[q].kernel, recs[q].level, ms};
      prev = recs[q].ev;
    }
  } else {
    cuda_fail(P, e, "hz_profile_graph");
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (g) cudaGraphDestroy(g);
  for (auto& r : recs) cudaEventDestroy(r.ev);
  cudaEventDestroy(start);
  return count;
}

// ------------------------------------------------------------------ groups of problems

struct hz_group {
  std::vector<hz_problem*> probs;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  int total = 0;
  cudaGraphExec_t graph = nullptr;
  std::string err;
};

static void group_release(hz_group* g) {
  if (g->graph) cudaGraphExecDestroy(g->graph);
  for (auto e : g->join) if (e) cudaEventDestroy(e);
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->stream) cudaStreamDestroy(g->stream);
}

#define GK(call)                                                  \
  do {                                                            \
    cudaError_t e__ = (call);                                     \
    if (e__ != cudaSuccess) {                                     \
      g->err = std::string(#call) + ": " + cudaGetErrorString(e__); \
      return HZ_ECUDA;                                            \
    }                                                             \
  } while (0)

hz_status hz_group_create(hz_problem* const* probs, int count, hz_group** out) {
  if (!out || !probs || count < 1 || count > LOOP_MAX_PROBLEMS) return HZ_EINVAL;
  *out = nullptr;
  hz_group* g = new hz_group();
  for (int i = 0; i < count; ++i) {
    if (!probs[i] || !probs[i]->setup) { delete g; return HZ_EINVAL; }
    g->probs.push_back(probs[i]);
    g->total += probs[i]->plan.batch;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming);
  g->join.assign(count, nullptr);
  for (int i = 0; i < count && !e; ++i) e = cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming);
  if (e) {
    group_release(g);
    delete g;
    return HZ_ECUDA;
  }
  *out = g;
  return HZ_OK;
}

// The group's solve graph: the WHILE loop's body holds one iteration of every problem, each on
// its own branch between a fork and a join; the control kernel watches every instance of every
// problem (the loop counter lives in the first problem's status block).
static hz_status group_graph(hz_group* g) {
  if (g->graph) {
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  LoopCtl ctl{};
  ctl.counter = loop_counter(g->probs[0]);
  ctl.problems = (int)g->probs.size();
  for (size_t i = 0; i < g->probs.size(); ++i) {
    ctl.st[i] = g->probs[i]->kv.st;
    ctl.batch[i] = g->probs[i]->plan.batch;
  }
  auto body = [&]() -> cudaError_t {
    cudaError_t e = cudaEventRecord(g->fork, g->stream);
    for (size_t i = 0; i < g->probs.size() && !e; ++i) {
      hz_problem* P = g->probs[i];
      e = cudaStreamWaitEvent(P->stream, g->fork, 0);
      if (!e) e = enqueue_iteration(P);
      if (!e) e = cudaEventRecord(g->join[i], P->stream);
      if (!e) e = cudaStreamWaitEvent(g->stream, g->join[i], 0);
    }
    return e;
  };
  cudaError_t e = build_loop_graph(g->stream, ctl, body, &g->graph);
  if (e) {
    g->err = std::string("building the group solve graph: ") + cudaGetErrorString(e);
    return HZ_ECUDA;
  }
  return HZ_OK;
}

hz_status hz_group_solve(hz_group* g, const double* const* rhs, double* const* x, double tol, int maxit,
                         hz_solve_info* infos) {
  if (!g || !rhs || !x || !(tol > 0) || maxit < 1) return HZ_EINVAL;
  if (maxit > HIST_CAP / 2 - 1) maxit = HIST_CAP / 2 - 1;
  const size_t np = g->probs.size();
  // every problem works on its own rhs and x buffers (copied in and out), so the group graph is
  // built once
  for (size_t i = 0; i < np; ++i) {
    if (!rhs[i] || !x[i] || (const double*)x[i] == rhs[i]) return HZ_EINVAL;
    hz_problem* P = g->probs[i];
    if (P->run.phase != hz_problem::Run::IDLE) return HZ_EINVAL;
    P->kv.b = P->b_int;
    P->kv.x = P->x_int;
  }
  if (!g->graph) {
    hz_status st = group_graph(g);
    if (st) return st;
  }
  // order after the callers' streams, then the start-up of every problem
  for (size_t i = 0; i < np; ++i) {
    hz_problem* P = g->probs[i];
    GK(cudaEventRecord(P->ev_in, P->user_stream));
    GK(cudaStreamWaitEvent(g->stream, P->ev_in, 0));
  }
  GK(cudaEventRecord(g->fork, g->stream));
  for (size_t i = 0; i < np; ++i) {
    hz_problem* P = g->probs[i];
    GK(cudaStreamWaitEvent(P->stream, g->fork, 0));
    GK(cudaMemcpyAsync(P->b_int, rhs[i], sizeof(double2) * (size_t)P->kv.N * P->plan.batch,
                       cudaMemcpyDeviceToDevice, P->stream));
    GK(launch_k_init(P->kv, tol, maxit, HIST_CAP, P->stream));
    GK(cudaEventRecord(g->join[i], P->stream));
    GK(cudaStreamWaitEvent(g->stream, g->join[i], 0));
  }
  int restarts = 0;
  for (;;) {
    // every iteration of every problem: one graph launch with a device-side loop
    GK(cudaGraphLaunch(g->graph, g->stream));
    // true residuals and final states
    GK(cudaEventRecord(g->fork, g->stream));
    for (size_t i = 0; i < np; ++i) {
      hz_problem* P = g->probs[i];
      GK(cudaStreamWaitEvent(P->stream, g->fork, 0));
      GK(launch_k_update_x(P->kv, false, P->stream));  // the last steps' pending solution update
      GK(launch_k_update_x(P->kv, true, P->stream));
      GK(launch_k_true_residual(P->kv, P->stream));
      GK(cudaMemcpyAsync(P->kstate_host, P->kv.st, sizeof(KState) * P->plan.batch, cudaMemcpyDeviceToHost, P->stream));
    }
    for (size_t i = 0; i < np; ++i) GK(cudaStreamSynchronize(g->probs[i]->stream));
    bool restarted = false;
    if (restarts < 8) {
      for (size_t i = 0; i < np; ++i) {
        hz_problem* P = g->probs[i];
        for (int b = 0; b < P->plan.batch; ++b) {
          const KState& hs = P->kstate_host[b];
          if (hs.done == 1 && hs.bnorm2 > 0 && !(hs.trr <= hs.tol2) && hs.it < maxit) {
            GK(launch_k_restart(instance_of(P->kv, b), P->stream));
            restarted = true;
          }
        }
        GK(cudaEventRecord(g->join[i], P->stream));
        GK(cudaStreamWaitEvent(g->stream, g->join[i], 0));
      }
    }
    if (!restarted) break;
    ++restarts;
  }
  for (size_t i = 0; i < np; ++i) {
    hz_problem* P = g->probs[i];
    GK(cudaMemcpyAsync(x[i], P->x_int, sizeof(double2) * (size_t)P->kv.N * P->plan.batch, cudaMemcpyDeviceToDevice,
                       P->stream));
    GK(cudaStreamSynchronize(P->stream));
  }
  hz_status worst = HZ_OK;
  int q = 0;
  for (size_t i = 0; i < np; ++i) {
    hz_problem* P = g->probs[i];
    for (int b = 0; b < P->plan.batch; ++b, ++q) {
      const KState& hs = P->kstate_host[b];
      double it = 0;
      hz_status sb = instance_status(hs, maxit, &it);
      if (sb != HZ_OK && worst == HZ_OK) worst = sb;
      if (infos) {
        infos[q].iterations = it;
        infos[q].relres_true = hs.bnorm2 > 0 ? std::sqrt(hs.trr / hs.bnorm2) : 0.0;
        infos[q].history_len = 0;
        infos[q].status = sb;
        infos[q].restarts = restarts + hs.shadow_restarts;
      }
    }
  }
  return worst;
}

const char* hz_group_last_error(const hz_group* g) { return g ? g->err.c_str() : "null group"; }

void hz_group_destroy(hz_group* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  group_release(g);
  delete g;
}

hz_status hz_set_stall_detection(hz_problem* P, double cos2, double step2, int max_restarts) {
  if (!P) return HZ_EINVAL;
  if (!(cos2 >= 0.0) || !(step2 >= 0.0) || !std::isfinite(cos2) || !std::isfinite(step2) || max_restarts < 0 ||
      max_restarts > 1024)
    return fail(P, HZ_EINVAL, "stall detection: thresholds must be finite and >= 0, max_restarts in [0, 1024]");
  P->kv.stall_cos2 = cos2;
  P->kv.stall_step2 = step2;
  P->kv.max_shadow_restarts = max_restarts;
  return HZ_OK;
}

const char* hz_kernel_name(int k) {
  static const char* names[] = {"gs_first", "gs_colour", "kacz_colour", "zero", "restrict_residual", "prolong_add",
                                "coarse_solve", "export", "k_update_p", "k_apply_rv", "k_update_s",
                                "k_apply_ts", "k_update_r", "smooth_restrict", "prolong_smooth", "kacz_level",
                                "kacz_sweep", "coarse_tail", "kacz_cluster", "jacobi", "kacz_grid", "k_update_x"};
  return (k >= 0 && k < HZ_K_COUNT) ? names[k] : "unknown";
}

int hz_krylov_scalars(hz_problem* P, int instance, double* out) {
  if (!P || !P->setup || !out || instance < 0 || instance >= P->plan.batch) return -1;
  KState ks;
  if (cudaMemcpy(&ks, P->kv.st + instance, sizeof(KState), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  const double v[17] = {ks.rho.x, ks.rho.y, ks.alpha.x, ks.alpha.y, ks.omega.x, ks.omega.y, ks.beta.x, ks.beta.y,
                        ks.rr, ks.ss, ks.tt, ks.bnorm2, (double)ks.it, (double)ks.done, ks.min_cos2,
                        (double)ks.shadow_restarts, ks.min_step2};
  for (int q = 0; q < 17; ++q) out[q] = v[q];
  return 17;
}

const char* hz_last_error(const hz_problem* P) { return P ? P->err.c_str() : "null problem"; }

const char* hz_status_string(int s) {
  switch (s) {
    case HZ_OK: return "HZ_OK";
    case HZ_EINVAL: return "HZ_EINVAL";
    case HZ_ENOMEM: return "HZ_ENOMEM";
    case HZ_ECUDA: return "HZ_ECUDA";
    case HZ_ENOTSETUP: return "HZ_ENOTSETUP";
    case HZ_EBREAKDOWN: return "HZ_EBREAKDOWN";
    case HZ_EMAXIT: return "HZ_EMAXIT";
    case HZ_ENONFINITE: return "HZ_ENONFINITE";
    case HZ_ETIMEOUT: return "HZ_ETIMEOUT";
    default: return "unknown";
  }
}

// ---------------------------------------------------------------- ray correction (Sec. 6, Table 7)

// The ray grid factor of the reading: the largest power of two with k m h <= 2.5 that divides n
// and leaves at least two ray cells.
static int ray_rule(int n, double k) {
  int m = 1;
  while (n % (2 * m) == 0 && n / (2 * m) >= 2 && k * (2 * m) / n <= 2.5 * (1 + 1e-12)) m *= 2;
  return m;
}

// Carves the ray correction's arrays out of `base` (null: sizes only); returns the bytes.
static size_t ray_layout(int n, int m, RayBlocks* B, double2** ph, unsigned char* base) {
  const int Nr = n / m + 1, Bs = 8 * Nr;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  const size_t blk = sizeof(double2) * (size_t)Bs * Bs * Nr, vec = sizeof(double2) * (size_t)Bs * Nr;
  B->n = n;
  B->m = m;
  B->Nr = Nr;
  B->Bs = Bs;
  B->L = (double2*)take(blk);
  B->D = (double2*)take(blk);
  B->U = (double2*)take(blk);
  B->Sinv = (double2*)take(blk);
  B->G = (double2*)take(blk);
  B->W = (double2*)take(blk);
  B->g = (double2*)take(vec);
  B->z = (double2*)take(vec);
  B->y = (double2*)take(vec);
  B->e = (double2*)take(vec);
  B->dz = (double2*)take(vec);
  B->fcol = (double2*)take(sizeof(double2) * Bs);
  B->perm = (int*)take(sizeof(int) * Bs);
  B->status = (int*)take(sizeof(int));
  *ph = (double2*)take(sizeof(double2) * 8 * (size_t)(n + 1) * (n + 1));
  return off;
}

static hz_status ray_build(hz_ray* R) {
  hz_problem* P = R->P;
  const RayBlocks& B = R->B;
  cudaStream_t s = P->stream;
  const auto t0 = std::chrono::steady_clock::now();
  const size_t blk = sizeof(double2) * (size_t)B.Bs * B.Bs * B.Nr;
  CK(cudaMemsetAsync(B.L, 0, blk, s));
  CK(cudaMemsetAsync(B.D, 0, blk, s));
  CK(cudaMemsetAsync(B.U, 0, blk, s));
  CK(cudaMemsetAsync(B.status, 0, sizeof(int), s));
  CK(launch_ray_phases(R->ph, P->n, R->k, s));
  CK(launch_ray_assemble(B, R->ph, P->kh64, s));
  CK(ray_factor(B, s));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, B.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return fail(P, HZ_EBREAKDOWN, "ray correction: a pivot block of P^H A P is singular");
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const cudaError_t ec = ray_coarse_solve(B, B.z, B.g, s);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (ec != cudaSuccess) e = ec;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&R->solve_graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(P, e, "capture of the ray solve");
  R->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return HZ_OK;
}

// x += P (P^H A P)^{-1} P^H r through the internal vectors and the captured solve.
static cudaError_t ray_apply(hz_ray* R, double2* x, const double2* r) {
  cudaStream_t s = R->P->stream;
  cudaError_t e = launch_ray_restrict(R->B.g, r, R->ph, R->B.n, R->B.m, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(R->solve_graph, s);
  if (e == cudaSuccess) e = launch_ray_prolong_add(x, R->B.z, R->ph, R->B.n, R->B.m, s);
  return e;
}

int hz_ray_spacing(int n, double k_ref) {
  if (n < 2 || !(k_ref > 0) || !std::isfinite(k_ref)) return 0;
  return ray_rule(n, k_ref);
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
static bool bytes_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

static bool ray_factor_ok(int n, int m) { return n >= 2 && m >= 1 && !(m & (m - 1)) && n % m == 0 && n / m <= HZ_RAY_MAX_NC; }

size_t hz_ray_footprint_bytes(int n, double k_ref, int m) {
  if (m == 0) m = hz_ray_spacing(n, k_ref);
  if (!ray_factor_ok(n, m)) return 0;
  RayBlocks B;
  double2* ph = nullptr;
  return ray_layout(n, m, &B, &ph, nullptr);
}

hz_status hz_ray_create(hz_problem* P, double k_ref, int m, void* arena, size_t arena_bytes, hz_ray** out) {
  if (!P || !out) return HZ_EINVAL;
  *out = nullptr;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!(k_ref > 0) || !std::isfinite(k_ref)) return fail(P, HZ_EINVAL, "ray correction: k_ref must be positive and finite");
  const int n = P->n;
  if (m == 0) m = ray_rule(n, k_ref);
  if (!ray_factor_ok(n, m))
    return fail(P, HZ_EINVAL, "ray correction: m must be a power of two dividing n with n / m <= HZ_RAY_MAX_NC");
  RayBlocks B0;
  double2* ph0 = nullptr;
  const size_t need = ray_layout(n, m, &B0, &ph0, nullptr);
  if (arena && arena_bytes < need) return fail(P, HZ_ENOMEM, "ray arena smaller than hz_ray_footprint_bytes");
  if (arena && ((uintptr_t)arena & 255)) return fail(P, HZ_EINVAL, "ray arena must be 256-byte aligned");
  StreamScope scope(P);
  hz_ray* R = new hz_ray;
  R->P = P;
  R->k = k_ref;
  R->bytes = need;
  if (arena) {
    R->mem = arena;
  } else if (cudaMalloc(&R->mem, R->bytes) != cudaSuccess) {
    cudaGetLastError();
    delete R;
    return fail(P, HZ_ENOMEM, "ray correction: device allocation refused");
  } else {
    R->own_mem = true;
  }
  ray_layout(n, m, &R->B, &R->ph, (unsigned char*)R->mem);
  const hz_status st = ray_build(R);
  if (st != HZ_OK) {
    hz_ray_destroy(R);
    return st;
  }
  *out = R;
  return HZ_OK;
}

hz_status hz_ray_get_info(const hz_ray* R, hz_ray_info* info) {
  if (!R || !info) return HZ_EINVAL;
  info->m = R->B.m;
  info->nc = R->B.Nr - 1;
  info->unknowns = R->B.Bs * R->B.Nr;
  info->kH = R->k * R->B.m / R->B.n;
  info->bytes = R->bytes;
  info->setup_ms = R->setup_ms;
  return HZ_OK;
}

hz_status hz_ray_restrict(hz_ray* R, const double* res, double* g) {
  if (!R) return HZ_EINVAL;
  hz_problem* P = R->P;
  const size_t fb = sizeof(double2) * (size_t)(R->B.n + 1) * (R->B.n + 1), rb = sizeof(double2) * (size_t)R->B.Bs * R->B.Nr;
  if (!res || !g || bytes_overlap(g, rb, res, fb)) return fail(P, HZ_EINVAL, "bad ray restriction arguments");
  StreamScope scope(P);
  CK(launch_ray_restrict((double2*)g, (const double2*)res, R->ph, R->B.n, R->B.m, P->stream));
  return HZ_OK;
}

hz_status hz_ray_coarse_solve(hz_ray* R, const double* g, double* z) {
  if (!R) return HZ_EINVAL;
  hz_problem* P = R->P;
  const size_t rb = sizeof(double2) * (size_t)R->B.Bs * R->B.Nr;
  if (!g || !z || bytes_overlap(z, rb, g, rb)) return fail(P, HZ_EINVAL, "bad ray solve arguments");
  StreamScope scope(P);
  const size_t bytes = sizeof(double2) * (size_t)R->B.Bs * R->B.Nr;
  CK(cudaMemcpyAsync(R->B.g, g, bytes, cudaMemcpyDeviceToDevice, P->stream));
  CK(cudaGraphLaunch(R->solve_graph, P->stream));
  CK(cudaMemcpyAsync(z, R->B.z, bytes, cudaMemcpyDeviceToDevice, P->stream));
  return HZ_OK;
}

hz_status hz_ray_blocks(hz_ray* R, double* lower, double* diag, double* upper) {
  if (!R) return HZ_EINVAL;
  hz_problem* P = R->P;
  StreamScope scope(P);
  const size_t blk = sizeof(double2) * (size_t)R->B.Bs * R->B.Bs * R->B.Nr;
  if (lower) CK(cudaMemcpyAsync(lower, R->B.L, blk, cudaMemcpyDeviceToDevice, P->stream));
  if (diag) CK(cudaMemcpyAsync(diag, R->B.D, blk, cudaMemcpyDeviceToDevice, P->stream));
  if (upper) CK(cudaMemcpyAsync(upper, R->B.U, blk, cudaMemcpyDeviceToDevice, P->stream));
  return HZ_OK;
}

hz_status hz_ray_correct(hz_ray* R, const double* res, double* x) {
  if (!R) return HZ_EINVAL;
  hz_problem* P = R->P;
  const size_t fb = sizeof(double2) * (size_t)(R->B.n + 1) * (R->B.n + 1);
  if (!res || !x || bytes_overlap(x, fb, res, fb)) return fail(P, HZ_EINVAL, "bad ray correction arguments");
  StreamScope scope(P);
  CK(ray_apply(R, (double2*)x, (const double2*)res));
  return HZ_OK;
}

void hz_ray_destroy(hz_ray* R) {
  if (!R) return;
  if (R->solve_graph) cudaGraphExecDestroy(R->solve_graph);
  if (R->own_mem) cudaFree(R->mem);  // waits for the device; touches no stream of the problem
  else if (R->mem) cudaDeviceSynchronize();  // the caller's arena may be reused once this returns
  delete R;
}

static hz_status cycle_run(hz_problem* P, hz_ray* R, const double2* b, double2* x, double tol, int maxc,
                           double* history, int history_cap, hz_solve_info* info, unsigned char* mem) {
  const long long N = (long long)(P->n + 1) * (P->n + 1);
  cudaStream_t s = P->stream;
  double2* r = (double2*)mem;
  double2* v = r + N;
  double2* z = v + N;
  double* partials = (double*)(z + N);
  double* nrm = partials + ray_reduction_blocks();
  const double n2 = (double)P->n * P->n;
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * N, s));
  CK(launch_ray_residual_norm(nullptr, b, nullptr, N, partials, nrm, s));
  double b2 = 0, rr = 0;
  CK(cudaMemcpyAsync(&b2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  hz_status st = b2 > 0 ? HZ_EMAXIT : HZ_OK;
  int cycles = 0, hl = 0;
  while (st == HZ_EMAXIT && cycles < maxc) {
    ++cycles;
    CK(launch_apply_fp64(v, x, P->kh64, P->n, 0.0, n2, s));
    CK(launch_ray_residual_norm(r, b, v, N, partials, nrm, s));
    const hz_status vs = vcycle_dev(P, (const double*)r, (double*)z);
    if (vs != HZ_OK) return vs;
    CK(launch_ray_axpy(x, z, N, s));
    if (R) {
      CK(launch_apply_fp64(v, x, P->kh64, P->n, 0.0, n2, s));
      CK(launch_ray_residual_norm(r, b, v, N, partials, nrm, s));
      CK(ray_apply(R, x, r));
    }
    CK(launch_apply_fp64(v, x, P->kh64, P->n, 0.0, n2, s));
    CK(launch_ray_residual_norm(r, b, v, N, partials, nrm, s));
    double r2 = 0;
    CK(cudaMemcpyAsync(&r2, nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rr = std::sqrt(r2 / b2);
    if (history && hl < history_cap) history[hl] = rr;
    ++hl;
    if (!std::isfinite(rr)) st = HZ_ENONFINITE;
    else if (rr <= tol) st = HZ_OK;
    else if (rr > 1e8) break;  // diverged: reported as HZ_EMAXIT
  }
  if (info) {
    info->iterations = cycles;
    info->relres_true = rr;
    info->history_len = std::min(hl, history_cap > 0 ? history_cap : 0);
    info->status = st;
    info->restarts = 0;
  }
  if (st == HZ_EMAXIT) return fail(P, st, rr > 1e8 ? "cycle solver diverged" : "cycle solver: maxc cycles without reaching tol");
  if (st == HZ_ENONFINITE) return fail(P, st, "cycle solver: non-finite residual");
  return HZ_OK;
}

size_t hz_cycle_scratch_bytes(int n) {
  if (n < 2 || n > 32768) return 0;
  const size_t N = (size_t)(n + 1) * (n + 1);
  return 3 * sizeof(double2) * N + sizeof(double) * (ray_reduction_blocks() + 2);
}

hz_status hz_cycle_solve(hz_problem* P, hz_ray* R, const double* rhs, double* x, double tol, int maxc, void* scratch,
                         size_t scratch_bytes, double* history, int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (P->plan.batch != 1) return fail(P, HZ_EINVAL, "batched hierarchy: the cycle solver takes one right-hand side");
  const size_t fb = sizeof(double2) * (size_t)(P->n + 1) * (P->n + 1);
  const size_t need = hz_cycle_scratch_bytes(P->n);
  if (!rhs || !x || bytes_overlap(x, fb, rhs, fb) || maxc < 1 || !(tol >= 0))
    return fail(P, HZ_EINVAL, "bad cycle-solve arguments");
  if (scratch && (bytes_overlap(scratch, need, x, fb) || bytes_overlap(scratch, need, rhs, fb)))
    return fail(P, HZ_EINVAL, "cycle-solve scratch overlaps rhs or x");
  if (R && R->P != P) return fail(P, HZ_EINVAL, "ray correction built for another problem");
  if (scratch && scratch_bytes < need) return fail(P, HZ_ENOMEM, "scratch smaller than hz_cycle_scratch_bytes");
  if (scratch && ((uintptr_t)scratch & 255)) return fail(P, HZ_EINVAL, "scratch must be 256-byte aligned");
  StreamScope scope(P);
  unsigned char* mem = (unsigned char*)scratch;
  if (!mem && cudaMalloc(&mem, need) != cudaSuccess) {
    cudaGetLastError();
    return fail(P, HZ_ENOMEM, "cycle solver: scratch allocation refused");
  }
  const hz_status st = cycle_run(P, R, (const double2*)rhs, (double2*)x, tol, maxc, history, history_cap, info, mem);
  if (!scratch) {
    cudaStreamSynchronize(P->stream);
    cudaFree(mem);
  }
  return st;
}

void hz_destroy(hz_problem* P) {
  if (!P) return;
  release(P);
  delete P;
}

}  // extern "C"
