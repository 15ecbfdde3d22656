// C ABI (include/hz.h): problem set-up, the level hierarchy of Sec. 5, the V-cycle driver, the
// graph-replayed Bi-CGSTAB loop of Sec. 6, and the step entry points used by the tests.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "hz_internal.h"

using namespace hz;

namespace {

constexpr int HIST_CAP = 32768;       // device history entries (two per iteration)
constexpr int MAX_COARSE_UNKNOWNS = 1089;
constexpr int PARTIAL_SLOTS = 4;
constexpr int MAX_G = 16384;
constexpr unsigned long long SHADOW_SEED = 0x5EED1312ull;
constexpr int PIPELINE = 3;  // iterations queued ahead of the convergence poll

// Scale bins in c = k_ref H: geometric midpoints between the paper's scales 0.3125, 0.625, 1.25
// and 2.5 (Sec. 4-5), and the guard band 1 < kH < 2 sqrt 2 for L relaxation.
const double BIN_LO = 0.625 / std::sqrt(2.0);
const double BIN_MID = 0.625 * std::sqrt(2.0);
const double BIN_HI = 1.25 * std::sqrt(2.0);
const double GUARD_LO = 1.0;
const double GUARD_HI = 2.0 * std::sqrt(2.0);

struct Level {
  int n = 0, pitch = 0;
  double H = 0;
  int relax_op = HZ_OP_L, smoother = HZ_SMOOTH_GS, resid_op = HZ_OP_L, nu = 1;
  void* kh = nullptr;  // k H, real, working precision
  int pk = 0;
  void* u = nullptr;  // working precision complex
  void* f = nullptr;  // working precision complex (levels >= 1)
  void* u2 = nullptr; // result of the fused post-smoothing pass (levels >= 1)
};

struct Plan {
  int levels = 0;
  bool fp32 = false;
  std::vector<int> n, pitch;
  size_t total = 0;
  // offsets
  std::vector<size_t> off_kh, off_u, off_f, off_u2;
  size_t off_kh64 = 0, off_vec = 0, vec_bytes = 0, off_ainv = 0, off_work = 0, off_state = 0, off_partials = 0,
         off_hist = 0, off_status = 0;
  int nvec = 11;
  int m_coarse = 0;
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
    if (l > 0 || P->fp32) {  // level 0 in FP64 reads the FP64 k h array directly
      P->off_kh[l] = off;
      off = align256(off + cells * re);
    }
    P->off_u[l] = off;
    off = align256(off + cells * ce);
    if (l > 0) {
      P->off_f[l] = off;
      off = align256(off + cells * ce);
      P->off_u2[l] = off;  // out-of-place result of the fused post-smoothing pass
      off = align256(off + cells * ce);
    }
  }
  size_t N = (size_t)(n + 1) * (n + 1);
  P->off_kh64 = off;
  off = align256(off + N * 8);
  P->vec_bytes = align256(N * 16);
  P->off_vec = off;
  off += P->vec_bytes * P->nvec;
  P->m_coarse = (nc + 1) * (nc + 1);
  P->off_ainv = off;
  off = align256(off + (size_t)P->m_coarse * P->m_coarse * ce);
  P->off_work = off;
  off = align256(off + (size_t)P->m_coarse * P->m_coarse * 2 * 16);
  P->off_state = off;
  off = align256(off + sizeof(KState));
  P->off_partials = off;
  off = align256(off + (size_t)PARTIAL_SLOTS * MAX_G * 8);
  P->off_hist = off;
  off = align256(off + (size_t)HIST_CAP * 8);
  P->off_status = off;
  off = align256(off + 256);
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
  KrylovVecs kv{};
  double2* b_int = nullptr;  // host-buffer solve: rhs and x on the device
  double2* x_int = nullptr;
  int* poll_host = nullptr;  // pinned: PIPELINE slots of 4 ints (it, first, done, half)
  cudaEvent_t ev[PIPELINE]{};
  cudaGraphExec_t graph = nullptr;
  const double2* graph_b = nullptr;
  double2* graph_x = nullptr;
  int num_sms = 0;
  std::string err;
  // Measurement: when set, every launch is followed by an event on `stream` (hz_profile_iteration).
  struct ProfRec { int kernel, level; cudaEvent_t ev; };
  std::vector<ProfRec>* prof = nullptr;
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
    if (e == cudaSuccess) e = cudaEventRecord(ev, P->stream);
    if (e == cudaSuccess) P->prof->push_back({kernel, level, ev});
  }
  return e;
}

// Relaxation/residual roles of Sec. 5 for a non-coarsest level (the oracle's level_policy).
void level_roles(int variant, double c, const std::vector<double>& c_local, bool guard, Level* L) {
  bool kacz = (c >= BIN_MID && c < BIN_HI);
  L->smoother = kacz ? HZ_SMOOTH_KACZMARZ : HZ_SMOOTH_GS;
  if (variant == HZ_VAR_SL_PLAIN) {
    L->relax_op = HZ_OP_M; L->smoother = HZ_SMOOTH_GS; L->resid_op = HZ_OP_M;
    return;
  }
  if (variant == HZ_VAR_SL) { L->relax_op = HZ_OP_M; L->resid_op = HZ_OP_M; return; }
  if (variant == HZ_VAR_HLM) { L->relax_op = HZ_OP_L; L->resid_op = HZ_OP_L; return; }
  L->resid_op = HZ_OP_L;
  L->relax_op = (c >= BIN_LO && c < BIN_HI) ? HZ_OP_M : HZ_OP_L;
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

// A Gauss-Seidel level with one sweep each way runs as two fused tile passes (hz_fused.cu).
bool fused(const hz_problem* P, int l) {
  const Level& L = P->lv[l];
  return l < P->plan.levels - 1 && L.smoother == HZ_SMOOTH_GS && L.nu == 1;
}

// Where level l's result after post-relaxation lives (what level l-1 interpolates).
void* final_u(const hz_problem* P, int l) {
  return (l > 0 && fused(P, l)) ? P->lv[l].u2 : P->lv[l].u;
}

// Pre-relaxation from a zero guess on level l into lv[l].u and the restricted residual into
// level l+1's f.
cudaError_t level_down(hz_problem* P, int l, Src f, const int* stop) {
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
    return mark(P, launch_smooth_restrict(fp32, u, pu, C.f, C.pitch, f.f, f.pf, f.f64, kh, pk, L.n, bA, bB, stop, s),
                HZ_K_SMOOTH_RESTRICT, l);
  if (L.smoother == HZ_SMOOTH_GS) {
    if ((e = mark(P, launch_gs_first(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, 0, bA, stop, s), HZ_K_GS_FIRST, l))) return e;
    if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, 1, bA, stop, s), HZ_K_GS_COLOUR, l))) return e;
    for (int it = 1; it < L.nu; ++it)
      for (int c = 0; c < 2; ++c)
        if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, c, bA, stop, s), HZ_K_GS_COLOUR, l))) return e;
  } else {
    size_t ce = fp32 ? 8 : 16;
    if ((e = mark(P, cudaMemset2DAsync(u, (size_t)pu * ce, 0, (size_t)(L.n + 1) * ce, L.n + 1, s), HZ_K_ZERO, l))) return e;
    for (int it = 0; it < L.nu; ++it)
      for (int c = 0; c < 5; ++c)
        if ((e = mark(P, launch_kacz_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, c, bA, stop, s), HZ_K_KACZ_COLOUR, l))) return e;
  }
  return mark(P, launch_restrict_residual(fp32, C.f, C.pitch, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, bB, stop, s), HZ_K_RESTRICT, l);
}

// `sweeps` sweeps of the level's smoother on lv[l].u in place; post selects the ordering.
cudaError_t level_sweeps(hz_problem* P, int l, Src f, int sweeps, bool post, const int* stop) {
  const Level& L = P->lv[l];
  bool fp32 = P->plan.fp32;
  int pk;
  const void* kh = kh_of(P, l, &pk);
  double bA = op_beta(P, L.relax_op);
  cudaStream_t s = P->stream;
  void* u = L.u;
  int pu = L.pitch;
  cudaError_t e;
  for (int it = 0; it < sweeps; ++it) {
    if (L.smoother == HZ_SMOOTH_GS) {
      for (int q = 0; q < 2; ++q)
        if ((e = mark(P, launch_gs_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, post ? 1 - q : q, bA, stop, s),
                      HZ_K_GS_COLOUR, l)))
          return e;
    } else {
      for (int q = 0; q < 5; ++q)
        if ((e = mark(P, launch_kacz_colour(fp32, u, pu, f.f, f.pf, f.f64, kh, pk, L.n, post ? 4 - q : q, bA, stop, s),
                      HZ_K_KACZ_COLOUR, l)))
          return e;
    }
  }
  return cudaSuccess;
}

// Correction from level l+1 and post-relaxation of level l. The result goes to `out` (pitch po):
// on the finest level a double2 array, otherwise final_u(l).
cudaError_t level_up(hz_problem* P, int l, Src f, void* out, int po, const int* stop) {
  const Level& L = P->lv[l];
  const Level& C = P->lv[l + 1];
  bool fp32 = P->plan.fp32;
  const void* ec = final_u(P, l + 1);
  cudaError_t e;
  if (fused(P, l)) {
    int pk;
    const void* kh = kh_of(P, l, &pk);
    return mark(P, launch_prolong_smooth(fp32, out, po, l == 0, L.u, L.pitch, ec, C.pitch, f.f, f.pf, f.f64, kh, pk,
                                         L.n, op_beta(P, L.relax_op), stop, P->stream),
                HZ_K_PROLONG_SMOOTH, l);
  }
  if ((e = mark(P, launch_prolong_add(fp32, L.u, L.pitch, ec, C.pitch, L.n, stop, P->stream), HZ_K_PROLONG, l))) return e;
  if ((e = level_sweeps(P, l, f, L.nu, true, stop))) return e;
  if (l == 0)
    return mark(P, launch_export(fp32, (double2*)out, po, L.u, L.pitch, L.n, 1.0, stop, P->stream), HZ_K_EXPORT, 0);
  return cudaSuccess;
}

cudaError_t coarse(hz_problem* P, const int* stop) {
  const Level& C = P->lv.back();
  return mark(P, launch_coarse_solve(P->plan.fp32, C.u, C.pitch, C.f, C.pitch, P->ainvT, C.n, stop, P->stream), HZ_K_COARSE,
              P->plan.levels - 1);
}

Src level_src(const hz_problem* P, int l, const double2* f0) {
  return l == 0 ? Src{f0, P->n + 1, true} : Src{P->lv[l].f, P->lv[l].pitch, false};
}

// z = V-cycle(f0) with f0 already h^2-scaled (double2, pitch n+1); z double2, pitch n+1.
cudaError_t run_vcycle(hz_problem* P, const double2* f0, double2* z, const int* stop) {
  int L = P->plan.levels;
  cudaError_t e;
  for (int l = 0; l < L - 1; ++l)
    if ((e = level_down(P, l, level_src(P, l, f0), stop))) return e;
  if ((e = coarse(P, stop))) return e;
  for (int l = L - 2; l >= 0; --l) {
    void* out = l == 0 ? (void*)z : final_u(P, l);
    int po = l == 0 ? P->n + 1 : P->lv[l].pitch;
    if ((e = level_up(P, l, level_src(P, l, f0), out, po, stop))) return e;
  }
  return cudaSuccess;
}

// One Bi-CGSTAB iteration (two preconditioner applications, Sec. 6).
cudaError_t enqueue_iteration(hz_problem* P) {
  const KrylovVecs& k = P->kv;
  cudaStream_t s = P->stream;
  const int* stop = &k.st->done;
  cudaError_t e;
  if ((e = mark(P, launch_k_update_p(k, s), HZ_K_UPDATE_P, 0))) return e;
  if ((e = run_vcycle(P, k.p, k.y, stop))) return e;
  if ((e = mark(P, launch_k_apply_rv(k, s), HZ_K_APPLY_RV, 0))) return e;
  if ((e = mark(P, launch_k_update_s(k, s), HZ_K_UPDATE_S, 0))) return e;
  if ((e = mark(P, launch_k_x_half(k, s), HZ_K_X_HALF, 0))) return e;
  if ((e = run_vcycle(P, k.s, k.z, stop))) return e;
  if ((e = mark(P, launch_k_apply_ts(k, s), HZ_K_APPLY_TS, 0))) return e;
  return mark(P, launch_k_update_xr(k, s), HZ_K_UPDATE_XR, 0);
}

hz_status build_graph(hz_problem* P) {
  if (P->graph) {
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_iteration(P);
  cudaError_t e2 = cudaStreamEndCapture(P->stream, &g);
  if (e) return cuda_fail(P, e, "capture of one Bi-CGSTAB iteration");
  if (e2) return cuda_fail(P, e2, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&P->graph, g, 0);
  cudaGraphDestroy(g);
  if (e) return cuda_fail(P, e, "cudaGraphInstantiate");
  P->graph_b = P->kv.b;
  P->graph_x = P->kv.x;
  return HZ_OK;
}

hz_status solve_device(hz_problem* P, const double* rhs, double* x, double tol, int maxit, double* history,
                       int history_cap, hz_solve_info* info) {
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!rhs || !x || !(tol > 0) || maxit < 1) return fail(P, HZ_EINVAL, "bad solve arguments");
  if ((const double*)rhs == x) return fail(P, HZ_EINVAL, "rhs and x may not alias");
  if (maxit > HIST_CAP / 2 - 1) maxit = HIST_CAP / 2 - 1;
  P->kv.b = (const double2*)rhs;
  P->kv.x = (double2*)x;
  if (!P->graph || P->graph_b != P->kv.b || P->graph_x != P->kv.x) {
    hz_status st = build_graph(P);
    if (st) return st;
  }
  cudaStream_t s = P->stream;
  const KrylovVecs& k = P->kv;
  CK(launch_k_init(k, tol, maxit, HIST_CAP, s));
  int restarts = 0;
  int state[4] = {0, 0, 0, 0};
  for (;;) {
    // Replay iterations, polling the flags of the iteration PIPELINE-1 steps back.
    long long launched = 0, polled = 0;
    bool done = false;
    while (!done) {
      if (launched < (long long)maxit + 2) {
        CK(cudaGraphLaunch(P->graph, s));
        int slot = (int)(launched % PIPELINE);
        CK(cudaMemcpyAsync(P->poll_host + 4 * slot, &k.st->it, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(P->ev[slot], s));
        ++launched;
      }
      if (launched - polled >= PIPELINE || launched >= (long long)maxit + 2) {
        int slot = (int)(polled % PIPELINE);
        CK(cudaEventSynchronize(P->ev[slot]));
        std::memcpy(state, P->poll_host + 4 * slot, sizeof(state));
        ++polled;
        if (state[2] != 0) done = true;
        else if (polled >= launched && launched >= (long long)maxit + 2) done = true;
      }
    }
    CK(cudaStreamSynchronize(s));
    KState hs;
    CK(cudaMemcpyAsync(&hs, k.st, sizeof(KState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs.done == 1 && hs.bnorm2 > 0) {
      CK(launch_k_true_residual(k, s));
      double trr = 0;
      CK(cudaMemcpyAsync(&trr, &k.st->trr, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (!(trr <= hs.tol2) && restarts < 8 && hs.it < maxit) {
        ++restarts;
        CK(launch_k_restart(k, s));
        continue;
      }
    } else if (hs.bnorm2 > 0) {
      CK(launch_k_true_residual(k, s));
      CK(cudaStreamSynchronize(s));
    }
    CK(cudaMemcpyAsync(&hs, k.st, sizeof(KState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    hz_status st = HZ_OK;
    double iters = hs.iters_x2 * 0.5;
    if (hs.done == 2) st = HZ_EBREAKDOWN;
    else if (hs.done == 3) st = HZ_ENONFINITE;
    else if (hs.done == 4 || hs.done == 0) { st = HZ_EMAXIT; iters = (double)maxit; }
    int hl = std::min(hs.hist_len, HIST_CAP);
    if (history && history_cap > 0 && hl > 0)
    {
      CK(cudaMemcpyAsync(history, k.hist, sizeof(double) * std::min(hl, history_cap), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    if (info) {
      info->iterations = iters;
      info->relres_true = hs.bnorm2 > 0 ? std::sqrt(hs.trr / hs.bnorm2) : 0.0;
      info->history_len = std::min(hl, history_cap > 0 ? history_cap : 0);
      info->status = st;
      info->restarts = restarts;
    }
    if (st == HZ_EBREAKDOWN) return fail(P, st, "Bi-CGSTAB breakdown");
    if (st == HZ_ENONFINITE) return fail(P, st, "non-finite value in the Krylov scalars");
    if (st == HZ_EMAXIT) return fail(P, st, "maximum iterations reached");
    return HZ_OK;
  }
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
      level_roles(o.variant, k_ref * L.H, c_local, o.guard != 0, &L);
      L.nu = L.smoother == HZ_SMOOTH_KACZMARZ ? o.nu_kacz : o.nu_gs;
    }
  }
  return true;
}

bool opts_ok(const hz_hierarchy_opts& o) {
  return !(o.variant < 0 || o.variant > 3 || (o.precision != 0 && o.precision != 1) || o.nu_gs < 1 || o.nu_gs > 8 ||
           o.nu_kacz < 1 || o.nu_kacz > 16 || o.k_ref < 0);
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
  for (auto& e : P->ev) if (e) { cudaEventDestroy(e); e = nullptr; }
  if (P->poll_host) { cudaFreeHost(P->poll_host); P->poll_host = nullptr; }
  if (P->ev_in) { cudaEventDestroy(P->ev_in); P->ev_in = nullptr; }
  if (P->ev_out) { cudaEventDestroy(P->ev_out); P->ev_out = nullptr; }
  if (P->stream) { cudaStreamSynchronize(P->stream); cudaStreamDestroy(P->stream); P->stream = nullptr; }
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
  CK(cudaMallocHost(&P->poll_host, sizeof(int) * 4 * PIPELINE));
  CK(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
  StreamScope scope(P);
  for (auto& e : P->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
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
    L.u2 = l > 0 ? (void*)(A + pl.off_u2[l]) : nullptr;
    int stride = 1 << l;
    if (L.kh) CK(launch_inject_kh(fp32, L.kh, L.pk, P->kh64, n, stride, L.n, (double)stride, s));
  }
  // Krylov vectors and scratch.
  KrylovVecs& k = P->kv;
  double2* vb = (double2*)(A + pl.off_vec);
  size_t stride_v = pl.vec_bytes / sizeof(double2);
  double2** slots[] = {&k.r, &k.rhat, &k.p, &k.v, &k.s, &k.t, &k.y, &k.z, &k.tr, &P->b_int, &P->x_int};
  for (int q = 0; q < pl.nvec; ++q) *slots[q] = vb + q * stride_v;
  k.x = nullptr;
  k.b = nullptr;
  k.kh = P->kh64;
  k.n = n;
  k.N = (long long)(n + 1) * (n + 1);
  k.scale_b = 1.0 / ((double)n * n);
  k.st = (KState*)(A + pl.off_state);
  k.partials = (double*)(A + pl.off_partials);
  k.hist = (double*)(A + pl.off_hist);
  long long want = (k.N + 255) / 256;
  k.G = (int)std::min<long long>(want, std::min(8LL * P->num_sms, (long long)MAX_G));
  if (k.G < 1) k.G = 1;
  CK(cudaMemsetAsync(k.st, 0, sizeof(KState), s));
  CK(launch_shadow(k.rhat, k.N, SHADOW_SEED, s));
  // Coarsest: dense inverse on the device.
  Level& C = P->lv.back();
  P->ainvT = A + pl.off_ainv;
  P->work = (double2*)(A + pl.off_work);
  P->status_dev = (int*)(A + pl.off_status);
  CK(launch_coarse_setup(fp32, P->ainvT, P->work, C.kh, C.pk, C.n, op_beta(P, C.relax_op), P->status_dev, s));
  int status = 1;
  CK(cudaMemcpyAsync(&status, P->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (status != 0) return fail(P, HZ_EINVAL, "coarsest operator is singular");
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
  return HZ_OK;
}

hz_status hz_vcycle(hz_problem* P, const double* r, double* z) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!r || !z || (const double*)r == z) return fail(P, HZ_EINVAL, "bad vcycle arguments");
  StreamScope scope(P);
  double h = 1.0 / P->n;
  CK(launch_import(false, P->kv.p, P->n + 1, (const double2*)r, P->n + 1, P->n, h * h, P->stream));
  CK(run_vcycle(P, P->kv.p, (double2*)z, nullptr));
  return HZ_OK;
}

hz_status hz_solve(hz_problem* P, const double* rhs, double* x, double tol, int maxit, double* history,
                   int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  StreamScope scope(P);
  return solve_device(P, rhs, x, tol, maxit, history, history_cap, info);
}

hz_status hz_solve_host(hz_problem* P, const double* rhs_host, double* x_host, double tol, int maxit,
                        double* history, int history_cap, hz_solve_info* info) {
  if (!P) return HZ_EINVAL;
  if (!P->setup) return fail(P, HZ_ENOTSETUP, "hz_setup_hierarchy has not been called");
  if (!rhs_host || !x_host) return fail(P, HZ_EINVAL, "null host pointer");
  StreamScope scope(P);
  size_t bytes = sizeof(double2) * (size_t)(P->n + 1) * (P->n + 1);
  CK(cudaMemcpyAsync(P->b_int, rhs_host, bytes, cudaMemcpyHostToDevice, P->stream));
  hz_status st = solve_device(P, (const double*)P->b_int, (double*)P->x_int, tol, maxit, history, history_cap, info);
  if (st != HZ_OK && st != HZ_EMAXIT && st != HZ_EBREAKDOWN && st != HZ_ENONFINITE) return st;
  CK(cudaMemcpyAsync(x_host, P->x_int, bytes, cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return st;
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
  if (level == 0) {
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
  P->graph_b = nullptr;  // the captured graph still refers to the previous buffers only by value
  return count;
}

const char* hz_kernel_name(int k) {
  static const char* names[] = {"gs_first", "gs_colour", "kacz_colour", "zero", "restrict_residual", "prolong_add",
                                "coarse_solve", "export", "k_update_p", "k_apply_rv", "k_update_s", "k_x_half",
                                "k_apply_ts", "k_update_xr", "smooth_restrict", "prolong_smooth"};
  return (k >= 0 && k < HZ_K_COUNT) ? names[k] : "unknown";
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

void hz_destroy(hz_problem* P) {
  if (!P) return;
  release(P);
  delete P;
}

}  // extern "C"
