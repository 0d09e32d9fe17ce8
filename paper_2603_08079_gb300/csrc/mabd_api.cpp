// Host side of the C ABI declared in include/mabd.h: scene validation,
// topology classification and ordering, prefactorization of the per-body
// system matrices (Eq. abd_final), device buffers and the kernel sequence of
// one step.  No C++ exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mabd.h"
#include "mabd_internal.h"
#include "principal_frame.h"
#include "topology.h"
#include "hbar_inv.h"

using namespace mabd;

namespace {

struct Rec {
  const char *name;
  cudaEvent_t a, b;
};

}  // namespace

struct mabd_ctx {
  mabd_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  bool frozen = false;
  bool cuda_failed = false;
  std::vector<mabd_body_desc> bodies;
  std::vector<mabd_joint_desc> joints;
  // bodies given with a non-diagonal second moment are kept in their
  // principal frame: caller's rest coordinates xbar = V xhat, A_lib = A V
  // (V row-major, 9 per body in user order; identity where has_frame is 0)
  std::vector<double> frames;
  std::vector<uint8_t> has_frame;
  bool any_frame = false;
  double *d_frames = nullptr;
  uint8_t *d_has_frame = nullptr;

  // ordering
  int32_t topology = MABD_TOPO_NONE;
  int32_t solver = MABD_SOLVER_AUTO;
  std::vector<int32_t> body_of_internal;   // internal -> user
  std::vector<int32_t> internal_of_body;   // user -> internal
  std::vector<int32_t> joint_of_internal;  // internal -> user
  std::vector<int32_t> internal_of_joint;  // user -> internal
  std::vector<int64_t> user_row_off;       // user joint -> first lambda row
  int64_t dual_rows = 0;

  // device memory
  std::vector<void *> allocs;
  int64_t device_bytes = 0;
  DevBodies B{};
  DevJoints J{};
  DevIncidence I{};
  DevChain C{};
  std::vector<CRLevel> levels;
  std::vector<CRLevelT<float>> levels_f;  // FP32 reduction of MABD_MIXED_FP32_DUAL
  // device copies of the level arrays and the first level of the single-CTA
  // tail of the reduction (levels.size() when the tail is off)
  CRLevel *d_levels = nullptr;
  CRLevelT<float> *d_levels_f = nullptr;
  int cr_tail_level = 0;
  // segment-tiled chain step of MABD_MIXED_FP32_DUAL (k_seg.cu), chosen with
  // MABD_CHAIN_SEG=1: tile levels (seg_lv[0]: the level-0 tiles of the
  // joints) and per-joint and per-body work arrays
  bool seg_on = false;
  int seg_up_t = SEG_UP_T;  // rows per tile of the upper systems (MABD_SEG_UP_T: a power of two)
  SegChain seg{};
  std::vector<SegLevel> seg_lv;
  DevTree T{};
  DevPCG P{};
  DevPCG32 P32{};
  int p32_nb[2] = {0, 0};  // blocks of the persistent FP32 solve (block Jacobi, learned); 0: off
  DevPCGN pn{};              // normalized-space solve of ball-joint graphs (k_pcgn.cu)
  int pn_nb[2] = {0, 0};     // its blocks (block Jacobi, learned); 0: off
  // learned preconditioner of the mixed PCG (joint graph, activations, weights)
  bool lpc_graph = false, lpc_on = false;
  LpcGraph lg{};
  LpcAct la{};
  LpcNet ln{};
  int lpc_fallbacks = 0;
  int pcg_last_iters = 0;
  double pcg_last_rel = 0.0;
  int *h_iter = nullptr;     // pinned [2]
  double *h_scal = nullptr;  // pinned [8]
  std::vector<int32_t> tree_lvl;  // level offsets (internal body order)
  std::vector<int32_t> tree_mid;  // per level: first leaf (bodies before it have children)
  std::vector<int8_t> tree_narrow;  // per level: its downward pass joins a single-block run
  DevForest F{};                       // the forest tree by tree (persistent kernel)
  DevTreeT<float> Tf{};                // FP32 elimination of the mixed tree form
  // loop solver: right-hand side and solution of a pass through the chain's
  // factors ([5][K]), and the chain's response at its two ends per breaker row
  double *loop_b = nullptr, *loop_x = nullptr, *loop_w = nullptr;
  int loop_rows = 0;  // rows of the loop breaker (3 or 5)
  int tree_mode = 0;                   // 0: level-scheduled launches; 128, 64 or 32: persistent kernel, threads
  double *cL = nullptr, *cR = nullptr, *Bn = nullptr;
  int *d_status = nullptr;
  unsigned long long *d_max = nullptr;
  int max_cap = 0;
  StepParams sp{};

  // pinned staging
  double *h_stage = nullptr;
  size_t h_stage_n = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
  // device-side state transfer: the caller's arrays as given, and the
  // internal -> user body map
  double *d_stage = nullptr;
  int32_t *d_boi = nullptr;
  int *d_flag = nullptr;

  // last CUDA failure (for mabd_error_detail)
  char err_detail[256] = {0};

  // CUDA graphs of one step (MABD_NO_GRAPHS=1 turns them off)
  bool graphs_off = false, graphs_built = false;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t g_step = nullptr, g_pre = nullptr, g_chunk = nullptr, g_post = nullptr;

  // MABD_DEBUG_SYNC=1: check every launch synchronously (diagnostics only)
  bool debug_sync = false;
  cudaError_t debug_err = cudaSuccess;

  // profiling
  bool prof_on = false;
  std::vector<Rec> recs;
  // profiling by graph replay: the step captured once with timing events
  // around every launch (external event-record nodes), replayed per step
  cudaGraphExec_t g_prof = nullptr;
  std::vector<Rec> prof_recs;
  bool prof_capture = false;
  cudaStream_t prof_stream = nullptr;
  std::map<std::string, std::pair<double, int64_t>> prof_acc;
};

namespace {

mabd_status cuda_fail_at(mabd_ctx *ctx, cudaError_t e, int line) {
  if (e == cudaSuccess) return MABD_OK;
  if (ctx && ctx->err_detail[0] == 0)
    std::snprintf(ctx->err_detail, sizeof(ctx->err_detail), "%s (%s) at mabd_api.cpp:%d",
                  cudaGetErrorName(e), cudaGetErrorString(e), line);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return MABD_ERR_OUT_OF_MEMORY;
  }
  if (ctx) ctx->cuda_failed = true;
  return MABD_ERR_CUDA;
}
#define cuda_fail(ctx, e) cuda_fail_at((ctx), (e), __LINE__)

#define CK(call)                                   \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e); \
  } while (0)

void *dalloc(mabd_ctx *ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void *p = nullptr;
  if (ctx->cfg.dev_alloc) {
    p = ctx->cfg.dev_alloc(bytes, ctx->cfg.alloc_user);
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) {
    ctx->allocs.push_back(p);
    ctx->device_bytes += (int64_t)bytes;
  }
  return p;
}

template <class T>
T *dnew(mabd_ctx *ctx, size_t n, bool &ok) {
  T *p = (T *)dalloc(ctx, n * sizeof(T));
  if (!p) ok = false;
  return p;
}

void free_all(mabd_ctx *ctx) {
  for (void *p : ctx->allocs) {
    if (ctx->cfg.dev_free) ctx->cfg.dev_free(p, ctx->cfg.alloc_user);
    else cudaFree(p);
  }
  ctx->allocs.clear();
  ctx->device_bytes = 0;
}

mabd_status map_status_bits(int bits) {
  if (bits & ST_INVERTED) return MABD_ERR_INVERTED;
  if (bits & ST_NONFINITE) return MABD_ERR_NONFINITE;
  if (bits & ST_NOT_SPD) return MABD_ERR_NOT_SPD;
  if (bits & (ST_POLAR_NOCONV | ST_PCG_NOCONV)) return MABD_ERR_NO_CONVERGENCE;
  if (bits & ST_TIMEOUT) return MABD_ERR_TIMEOUT;
  if (bits & ST_BOUNDS) return MABD_ERR_INVALID_ARG;
  return MABD_OK;
}

inline bool finite_arr(const double *a, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

inline int joint_rows(int type) { return joint_nrows(type); }

// --------------------------------------------------------------------------
// topology
// --------------------------------------------------------------------------
// the joint graph of the context's scene
Graph scene_graph(const mabd_ctx *ctx) {
  std::vector<uint8_t> fixed(ctx->bodies.size());
  for (size_t j = 0; j < fixed.size(); ++j) fixed[j] = ctx->bodies[j].fixed ? 1 : 0;
  const size_t K = ctx->joints.size();
  std::vector<int64_t> ja(K), jb(K);
  std::vector<int> jt(K);
  for (size_t k = 0; k < K; ++k) {
    ja[k] = ctx->joints[k].body_a;
    jb[k] = ctx->joints[k].body_b;
    jt[k] = ctx->joints[k].type;
  }
  return mabd::build_graph(fixed, ja, jb, jt);
}

// --------------------------------------------------------------------------
// per-body structured inverse of Hbar_A = M_A/h^2 + Kbar_A (Eq. abd_final)
// --------------------------------------------------------------------------
bool structured_hinv(const mabd_body_desc &d, double h, double out[HINV_N]) {
  const double s[3] = {d.second_moment[0], d.second_moment[1], d.second_moment[2]};
  return hbar_inverse(d.mass, s, d.volume, d.young, d.poisson, h, out);
}

// --------------------------------------------------------------------------
// profiling around launches
// --------------------------------------------------------------------------
// debug mode: report an error left pending by an earlier runtime call
void dbg_pending(const char *where) {
  static const bool on = [] {
    const char *d = std::getenv("MABD_DEBUG_SYNC");
    return d && d[0] == '1';
  }();
  if (!on) return;
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) std::fprintf(stderr, "mabd debug: pending %s at %s\n", cudaGetErrorName(e), where);
}

// an NVTX range over a launch group (host timeline of a profiler; a no-op
// without one)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <class F>
void run(mabd_ctx *ctx, const char *name, F &&f) {
  NvtxRange range(name);
  if (ctx->debug_sync) {
    cudaError_t e0 = cudaGetLastError();
    f();
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    cudaError_t e = e0 != cudaSuccess ? e0 : (e1 != cudaSuccess ? e1 : e2);
    if (e != cudaSuccess) {
      if (ctx->err_detail[0] == 0)
        std::snprintf(ctx->err_detail, sizeof(ctx->err_detail), "%s (%s) %s launch %s",
                      cudaGetErrorName(e), cudaGetErrorString(e),
                      e0 != cudaSuccess ? "before" : "in", name);
      std::fprintf(stderr, "mabd debug: %s\n", ctx->err_detail);
      ctx->debug_err = e;
    }
    return;
  }
  if (ctx->prof_capture) {
    // inside the capture of the profiling graph: event-record nodes
    Rec r{name, nullptr, nullptr};
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    cudaEventRecordWithFlags(r.a, ctx->prof_stream, cudaEventRecordExternal);
    f();
    cudaEventRecordWithFlags(r.b, ctx->prof_stream, cudaEventRecordExternal);
    ctx->prof_recs.push_back(r);
    return;
  }
  if (!ctx->prof_on) {
    f();
    return;
  }
  Rec r{name, nullptr, nullptr};
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  cudaEventRecord(r.a, ctx->stream);
  f();
  cudaEventRecord(r.b, ctx->stream);
  ctx->recs.push_back(r);
}

mabd_status harvest_profile(mabd_ctx *ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto &r : ctx->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto &acc = ctx->prof_acc[r.name];
    acc.first += ms;
    acc.second += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ctx->recs.clear();
  return MABD_OK;
}

mabd_status read_status(mabd_ctx *ctx) {
  int bits = 0;
  CK(cudaMemcpyAsync(&bits, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (bits) {
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return map_status_bits(bits);
}

mabd_status ensure_stage(mabd_ctx *ctx, size_t n) {
  if (ctx->stage_pending) {
    CK(cudaEventSynchronize(ctx->stage_done));
    ctx->stage_pending = false;
  }
  if (ctx->h_stage_n >= n) return MABD_OK;
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  ctx->h_stage = nullptr;
  ctx->h_stage_n = 0;
  CK(cudaMallocHost((void **)&ctx->h_stage, n * sizeof(double)));
  ctx->h_stage_n = n;
  return MABD_OK;
}

}  // namespace

// v in the principal frame of body j: V^T v (unchanged for bodies without one)
static void to_principal(const mabd_ctx *ctx, int64_t j, double v[3]) {
  if (j < 0 || !ctx->has_frame[j]) return;
  const double *V = ctx->frames.data() + 9 * j;
  const double x[3] = {v[0], v[1], v[2]};
  for (int c = 0; c < 3; ++c) v[c] = V[c] * x[0] + V[3 + c] * x[1] + V[6 + c] * x[2];
}

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

void mabd_config_default(mabd_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->h = 1e-2;
  cfg->gravity[2] = -9.8;
  cfg->precision = MABD_FP64;
  cfg->solver = MABD_SOLVER_AUTO;
  cfg->pcg_max_iters = 2000;
  cfg->pcg_rtol = 1e-13;
  cfg->refine_steps = 1;
  cfg->residual_rhs = 1;
}

const char *mabd_status_string(mabd_status s) {
  switch (s) {
    case MABD_OK: return "ok";
    case MABD_ERR_INVALID_ARG: return "invalid argument";
    case MABD_ERR_BAD_STATE: return "call out of order";
    case MABD_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MABD_ERR_CUDA: return "CUDA error (context unusable)";
    case MABD_ERR_NOT_SPD: return "matrix not positive definite";
    case MABD_ERR_INVERTED: return "inverted body (det A <= 0)";
    case MABD_ERR_NONFINITE: return "non-finite value";
    case MABD_ERR_NO_CONVERGENCE: return "iteration did not converge";
    case MABD_ERR_TIMEOUT: return "timeout";
    case MABD_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

mabd_status mabd_create(const mabd_config *cfg, mabd_ctx **out) {
  dbg_pending("enter mabd_create");
  if (!cfg || !out) return MABD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->h > 0.0) || !std::isfinite(cfg->h) || !finite_arr(cfg->gravity, 3))
    return MABD_ERR_INVALID_ARG;
  if (cfg->precision != MABD_FP64 && cfg->precision != MABD_MIXED && cfg->precision != MABD_MIXED_FP32_DUAL)
    return MABD_ERR_INVALID_ARG;
  if (cfg->refine_steps < 0 || cfg->refine_steps > MABD_MAX_REFINE) return MABD_ERR_INVALID_ARG;
  if (cfg->solver < MABD_SOLVER_AUTO || cfg->solver > MABD_SOLVER_LOOP) return MABD_ERR_INVALID_ARG;
  if (cfg->pcg_max_iters < 1 || !(cfg->pcg_rtol > 0.0)) return MABD_ERR_INVALID_ARG;
  if ((cfg->rotation_mode != MABD_ROTATION_POLAR && cfg->rotation_mode != MABD_ROTATION_NORMALIZED) ||
      (cfg->jacobian_mode != MABD_JACOBIAN_FROZEN && cfg->jacobian_mode != MABD_JACOBIAN_FULL))
    return MABD_ERR_INVALID_ARG;
  if ((cfg->dev_alloc == nullptr) != (cfg->dev_free == nullptr)) return MABD_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return MABD_ERR_CUDA;
  }
  mabd_ctx *ctx = new (std::nothrow) mabd_ctx();
  if (!ctx) return MABD_ERR_OUT_OF_MEMORY;
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cfg->stream;
  cudaGetDevice(&ctx->device);
  {
    const char *dbg = std::getenv("MABD_DEBUG_SYNC");
    ctx->debug_sync = dbg && dbg[0] == '1';
    const char *ng = std::getenv("MABD_NO_GRAPHS");
    ctx->graphs_off = ng && ng[0] == '1';
  }
  if (cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return MABD_ERR_CUDA;
  }
  *out = ctx;
  return MABD_OK;
}

mabd_status mabd_add_bodies(mabd_ctx *ctx, int64_t n, const mabd_body_desc *d, int64_t *first_id) {
  dbg_pending("enter mabd_add_bodies");
  if (!ctx || n < 0 || (n > 0 && !d)) return MABD_ERR_INVALID_ARG;
  if (ctx->frozen) return MABD_ERR_BAD_STATE;
  if ((int64_t)ctx->bodies.size() + n > (int64_t)INT32_MAX / 16) return MABD_ERR_INVALID_ARG;
  std::vector<mabd_body_desc> add(d, d + n);
  std::vector<double> fr(9 * (size_t)n, 0.0);
  std::vector<uint8_t> hf((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) {
    const auto &b = d[i];
    if (!(b.mass > 0.0) || !(b.volume > 0.0) || !(b.young > 0.0) || !(b.poisson >= 0.0) ||
        !(b.poisson < 0.5) || !std::isfinite(b.mass) || !std::isfinite(b.volume) ||
        !std::isfinite(b.young) || !finite_arr(b.second_moment, 6) || !finite_arr(b.q, 12) ||
        !finite_arr(b.qdot, 12) || (b.fixed != 0 && b.fixed != 1))
      return MABD_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
      if (!(b.second_moment[a] > 0.0)) return MABD_ERR_INVALID_ARG;
    const double tr = b.second_moment[0] + b.second_moment[1] + b.second_moment[2];
    double *V = fr.data() + 9 * i;
    V[0] = V[4] = V[8] = 1.0;
    bool diag = true;
    for (int a = 3; a < 6; ++a) diag = diag && std::fabs(b.second_moment[a]) <= 1e-12 * tr;
    if (diag) continue;
    // the principal frame: Sigma = V diag(w) V^T, xbar = V xhat, so the
    // body's affine matrix in that frame is A V (rest points, axes and
    // reference directions of its joints are turned by V^T at prefactor)
    double w[3];
    if (!sym3_eigen(b.second_moment, w, V) || !(w[0] > 0.0) || !(w[1] > 0.0) || !(w[2] > 0.0))
      return MABD_ERR_INVALID_ARG;
    auto &o = add[i];
    for (int a = 0; a < 3; ++a) o.second_moment[a] = w[a];
    for (int a = 3; a < 6; ++a) o.second_moment[a] = 0.0;
    frame_A(b.q, V, false, o.q);
    frame_A(b.qdot, V, false, o.qdot);
    hf[i] = 1;
  }
  if (first_id) *first_id = (int64_t)ctx->bodies.size();
  ctx->bodies.insert(ctx->bodies.end(), add.begin(), add.end());
  ctx->frames.insert(ctx->frames.end(), fr.begin(), fr.end());
  ctx->has_frame.insert(ctx->has_frame.end(), hf.begin(), hf.end());
  for (uint8_t f : hf) ctx->any_frame = ctx->any_frame || f;
  return MABD_OK;
}

mabd_status mabd_add_joints(mabd_ctx *ctx, int64_t n, const mabd_joint_desc *d, int64_t *first_id) {
  dbg_pending("enter mabd_add_joints");
  if (!ctx || n < 0 || (n > 0 && !d)) return MABD_ERR_INVALID_ARG;
  if (ctx->frozen) return MABD_ERR_BAD_STATE;
  if ((int64_t)ctx->joints.size() + n > (int64_t)INT32_MAX / 16) return MABD_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i) {
    const auto &j = d[i];
    if (j.type != MABD_JOINT_BALL && j.type != MABD_JOINT_HINGE && j.type != MABD_JOINT_UNIVERSAL &&
        j.type != MABD_JOINT_PRISMATIC)
      return MABD_ERR_INVALID_ARG;
    // a universal joint's fourth row lies on body b alone: b must be a body
    if (j.type == MABD_JOINT_UNIVERSAL && j.body_b < 0) return MABD_ERR_INVALID_ARG;
    if (!finite_arr(j.anchor_a, 3) || !finite_arr(j.anchor_b, 3) || !finite_arr(j.axis_a, 3) ||
        !finite_arr(j.axis_b, 3))
      return MABD_ERR_INVALID_ARG;
    if (j.type != MABD_JOINT_BALL) {
      double na = j.axis_a[0] * j.axis_a[0] + j.axis_a[1] * j.axis_a[1] + j.axis_a[2] * j.axis_a[2];
      double nb = j.axis_b[0] * j.axis_b[0] + j.axis_b[1] * j.axis_b[1] + j.axis_b[2] * j.axis_b[2];
      if (!(na > 0.0) || !(nb > 0.0) || !(j.axis_len > 0.0) || !std::isfinite(j.axis_len))
        return MABD_ERR_INVALID_ARG;
    }
    if (j.type == MABD_JOINT_PRISMATIC) {
      // reference directions: finite, non-zero, and ref_a not along axis_a
      if (!finite_arr(j.ref_a, 3) || !finite_arr(j.ref_b, 3)) return MABD_ERR_INVALID_ARG;
      const double *u = j.axis_a, *c = j.ref_a;
      const double nu = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      const double nc = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      const double cx = u[1] * c[2] - u[2] * c[1], cy = u[2] * c[0] - u[0] * c[2], cz = u[0] * c[1] - u[1] * c[0];
      const double nrb = std::sqrt(j.ref_b[0] * j.ref_b[0] + j.ref_b[1] * j.ref_b[1] + j.ref_b[2] * j.ref_b[2]);
      if (!(nc > 0.0) || !(nrb > 0.0) || !(std::sqrt(cx * cx + cy * cy + cz * cz) > 1e-6 * nu * nc))
        return MABD_ERR_INVALID_ARG;
    }
  }
  if (first_id) *first_id = (int64_t)ctx->joints.size();
  ctx->joints.insert(ctx->joints.end(), d, d + n);
  return MABD_OK;
}

}  // extern "C"

// The level-scheduled elimination of T: upward one launch per level,
// deepest first; downward root first, one launch per wide level and one
// single-block launch per run of consecutive narrow levels.  R(name,
// launch) issues a launch (the step wraps it for profiling).
template <typename S, typename R>
static void tree_levels(mabd_ctx *ctx, const DevTreeT<S> &T, cudaStream_t s, R &&runl) {
  const StepParams &p = ctx->sp;
  const auto &lv = ctx->tree_lvl;
  const auto &nw = ctx->tree_narrow;
  const int nl = (int)lv.size() - 1;
  for (int l = nl - 1; l >= 0; --l)
    runl("tree_up", [&] { launch_tree_up(ctx->B, ctx->J, T, lv[l], lv[l + 1], l == 0, p, ctx->d_status, s); });
  for (int l = 0; l < nl;) {
    if (nw[l]) {
      int lb = l + 1;
      while (lb < nl && nw[lb]) ++lb;
      runl("tree_down", [&] { launch_tree_down_run(ctx->B, ctx->J, T, l, lb, p, s); });
      l = lb;
    } else {
      runl("tree_down", [&] { launch_tree_down(ctx->B, ctx->J, T, lv[l], lv[l + 1], p, ctx->d_status, s); });
      ++l;
    }
  }
}

// Path of the tree elimination: one launch per level (upward deepest
// first, then downward), or the persistent forest kernel with one block of
// 128, 64 or 32 threads per tree (both passes in one launch).  The tuner runs
// the body and joint kernels on the initial state, then times each path on
// it (best of two CUDA-event timings; the downward pass moves the state, so
// it is saved and put back around every trial) and keeps the fastest.
// MABD_TREE_MODE=levels|forest128|forest64|forest32 forces the path.
template <typename S>
static mabd_status tune_tree_t(mabd_ctx *ctx, const DevTreeT<S> &TT) {
  const char *fm = std::getenv("MABD_TREE_MODE");
  if (fm) {
    ctx->tree_mode = std::strcmp(fm, "forest128") == 0 ? 128
                     : std::strcmp(fm, "forest64") == 0  ? 64
                     : std::strcmp(fm, "forest32") == 0  ? 32
                                                         : 0;
    return MABD_OK;
  }
  if (ctx->F.ntrees <= 0) return MABD_OK;
  cudaStream_t s = ctx->stream;
  const StepParams &p = ctx->sp;
  // inputs of the elimination in its precision
  if (sizeof(S) == 8) {
    launch_body_prep(ctx->B, p, ctx->d_status, s);
    launch_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s);
  } else {
    launch_mx_body_prep(ctx->B, p, ctx->d_status, s);
    launch_mx_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s);
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int M = ctx->B.M;
  double *sq = nullptr;
  CK(cudaMallocAsync((void **)&sq, 24 * (size_t)M * sizeof(double), s));
  CK(cudaMemcpyAsync(sq, ctx->B.q, 12 * (size_t)M * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(sq + 12 * (size_t)M, ctx->B.qd, 12 * (size_t)M * 8, cudaMemcpyDeviceToDevice, s));
  float best = 1e30f;
  for (int mode : {0, 128, 64, 32})
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(e0, s));
      if (mode == 0) {
        tree_levels(ctx, TT, s, [](const char *, auto &&f) { f(); });
      } else {
        launch_tree_forest(ctx->B, ctx->J, TT, ctx->F, p, ctx->d_status, s, mode);
      }
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        ctx->tree_mode = mode;
      }
      CK(cudaMemcpyAsync(ctx->B.q, sq, 12 * (size_t)M * 8, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(ctx->B.qd, sq + 12 * (size_t)M, 12 * (size_t)M * 8, cudaMemcpyDeviceToDevice, s));
    }
  CK(cudaFreeAsync(sq, s));
  CK(cudaStreamSynchronize(s));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  return MABD_OK;
}

static mabd_status tune_tree(mabd_ctx *ctx) {
  if (ctx->cfg.precision == MABD_MIXED_FP32_DUAL) return tune_tree_t<float>(ctx, ctx->Tf);
  return tune_tree_t<double>(ctx, ctx->T);
}

extern "C" {

mabd_status mabd_prefactor(mabd_ctx *ctx) {
  dbg_pending("enter mabd_prefactor");
  if (!ctx) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (ctx->frozen) return MABD_ERR_BAD_STATE;
  const int M = (int)ctx->bodies.size(), K = (int)ctx->joints.size();
  for (int k = 0; k < K; ++k) {
    const auto &j = ctx->joints[k];
    if (j.body_a < 0 || j.body_a >= M || j.body_b < MABD_WORLD || j.body_b >= M ||
        j.body_a == j.body_b)
      return MABD_ERR_INVALID_ARG;
    const bool afree = !ctx->bodies[j.body_a].fixed;
    const bool bfree = j.body_b >= 0 && !ctx->bodies[j.body_b].fixed;
    if (!afree && !bfree) return MABD_ERR_INVALID_ARG;  // no unknown: rows would be void
    if (j.type == MABD_JOINT_UNIVERSAL && !bfree) return MABD_ERR_INVALID_ARG;  // row 3 lies on b
  }
  // ---- topology and ordering
  Graph g = scene_graph(ctx);
  std::vector<int32_t> border, jorder, cborder, cjorder;
  TreeOrder tord;
  // the chain, tree and loop solvers take ball and hinge joints; a scene
  // with universal (4 rows) or prismatic joints (three point pairs) takes
  // the PCG solver
  bool pcg_only = false, has_prism = false;
  for (int k = 0; k < K; ++k) {
    pcg_only = pcg_only || g.jtype[k] == MABD_JOINT_UNIVERSAL || g.jtype[k] == MABD_JOINT_PRISMATIC;
    has_prism = has_prism || g.jtype[k] == MABD_JOINT_PRISMATIC;
  }
  // the paper's variants (Alg. 1, the full constraint gradient) exist in
  // the FP64 form; the full gradient's frame term is carried by the tree
  // and PCG solvers' kernels (the chain and loop solvers build their blocks
  // from point compliances), and needs a frame attached to one body
  const bool full_grad = ctx->cfg.jacobian_mode == MABD_JACOBIAN_FULL;
  if ((ctx->cfg.rotation_mode != MABD_ROTATION_POLAR || full_grad) && ctx->cfg.precision != MABD_FP64) {
    std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                  "MABD_ROTATION_NORMALIZED and MABD_JACOBIAN_FULL exist in the FP64 form only");
    return MABD_ERR_UNSUPPORTED;
  }
  if (full_grad)
    for (int k = 0; k < K; ++k)
      if (g.jtype[k] == MABD_JOINT_UNIVERSAL) {
        std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                      "MABD_JACOBIAN_FULL: the universal joint's frame follows both bodies");
        return MABD_ERR_UNSUPPORTED;
      }
  const bool is_chain = K > 0 && chain_order(g, cborder, cjorder);
  const bool is_tree = K > 0 && tree_order(g, tord);
  std::vector<int32_t> rborder, rjorder;
  const bool is_ring = K > 0 && !is_chain && !is_tree && ring_order(g, rborder, rjorder);
  int solver = ctx->cfg.solver;
  if (K == 0) {
    ctx->topology = MABD_TOPO_NONE;
    solver = MABD_SOLVER_AUTO;
  } else {
    ctx->topology = is_chain ? MABD_TOPO_CHAIN
                             : (is_tree ? MABD_TOPO_TREE : (is_ring ? MABD_TOPO_LOOP : MABD_TOPO_GRAPH));
    if (solver == MABD_SOLVER_AUTO)
      solver = is_chain ? MABD_SOLVER_CHAIN
                        : (is_tree ? MABD_SOLVER_TREE
                                   : ((is_ring && ctx->cfg.precision == MABD_FP64) ? MABD_SOLVER_LOOP
                                                                                   : MABD_SOLVER_PCG));
  }
  if (pcg_only && solver != MABD_SOLVER_PCG) {
    if (ctx->cfg.solver != MABD_SOLVER_AUTO) {
      std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                    "universal and prismatic joints are solved by the PCG solver only");
      return MABD_ERR_UNSUPPORTED;
    }
    solver = MABD_SOLVER_PCG;
  }
  if (full_grad && K > 0 && solver != MABD_SOLVER_PCG && solver != MABD_SOLVER_TREE) {
    if (ctx->cfg.solver != MABD_SOLVER_AUTO) {
      std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                    "MABD_JACOBIAN_FULL is solved by the tree or the PCG solver");
      return MABD_ERR_UNSUPPORTED;
    }
    solver = is_tree && !pcg_only ? MABD_SOLVER_TREE : MABD_SOLVER_PCG;
  }
  if (solver == MABD_SOLVER_CHAIN && !is_chain) return MABD_ERR_UNSUPPORTED;
  if (solver == MABD_SOLVER_TREE && !is_tree) return MABD_ERR_UNSUPPORTED;
  if (solver == MABD_SOLVER_LOOP && (!is_ring || ctx->cfg.precision != MABD_FP64)) {
    std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                  "the loop solver takes a single closed loop of bodies, in the FP64 form");
    return MABD_ERR_UNSUPPORTED;
  }
  if (ctx->cfg.precision == MABD_MIXED && K > 0 && solver == MABD_SOLVER_TREE) {
    std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                  "the mixed-precision form of the tree solver is MABD_MIXED_FP32_DUAL");
    return MABD_ERR_UNSUPPORTED;
  }
  if (solver == MABD_SOLVER_CHAIN) {
    border = cborder;
    jorder = cjorder;
  } else if (solver == MABD_SOLVER_LOOP) {
    border = rborder;
    jorder = rjorder;
  } else if (solver == MABD_SOLVER_TREE) {
    border = tord.border;
    jorder = tord.jorder;
  } else {
    border.resize(M);
    for (int j = 0; j < M; ++j) border[j] = j;
    jorder.resize(K);
    for (int k = 0; k < K; ++k) jorder[k] = k;
  }
  ctx->solver = solver;
  ctx->body_of_internal = border;
  ctx->internal_of_body.assign(M, -1);
  for (int i = 0; i < M; ++i) ctx->internal_of_body[border[i]] = i;
  ctx->joint_of_internal = jorder;
  ctx->internal_of_joint.assign(K, -1);
  for (int i = 0; i < K; ++i) ctx->internal_of_joint[jorder[i]] = i;
  ctx->user_row_off.assign(K + 1, 0);
  for (int k = 0; k < K; ++k) ctx->user_row_off[k + 1] = ctx->user_row_off[k] + joint_rows(ctx->joints[k].type);
  ctx->dual_rows = ctx->user_row_off[K];

  // ---- host arrays in internal order
  const double h = ctx->cfg.h;
  std::vector<double> q(12 * (size_t)M), qd(12 * (size_t)M), sig(3 * (size_t)M), mass(M), vmu(M),
      vlam(M), hinv(HINV_N * (size_t)M);
  std::vector<uint8_t> fixed(M);
  for (int i = 0; i < M; ++i) {
    const auto &d = ctx->bodies[border[i]];
    for (int c = 0; c < 12; ++c) {
      q[(size_t)c * M + i] = d.q[c];
      qd[(size_t)c * M + i] = d.qdot[c];
    }
    for (int a = 0; a < 3; ++a) sig[(size_t)a * M + i] = d.second_moment[a];
    mass[i] = d.mass;
    const double mu = d.young / (2.0 * (1.0 + d.poisson));
    const double lam = d.young * d.poisson / ((1.0 + d.poisson) * (1.0 - 2.0 * d.poisson));
    vmu[i] = d.volume * mu;
    vlam[i] = d.volume * lam;
    fixed[i] = d.fixed ? 1 : 0;
    double hv[HINV_N];
    if (!fixed[i]) {
      if (!structured_hinv(d, h, hv)) return MABD_ERR_NOT_SPD;
    } else {
      std::memset(hv, 0, sizeof(hv));
    }
    for (int c = 0; c < HINV_N; ++c) hinv[(size_t)c * M + i] = hv[c];
  }
  std::vector<int8_t> jtype(K);
  std::vector<int32_t> ja(K), jb(K);
  std::vector<uint8_t> jfl(K);
  std::vector<double> pa1(3 * (size_t)K), pb1(3 * (size_t)K), pa2(3 * (size_t)K), pb2(3 * (size_t)K),
      ua(3 * (size_t)K), pa3, pb3;
  if (has_prism) {
    pa3.assign(3 * (size_t)K, 0.0);
    pb3.assign(3 * (size_t)K, 0.0);
  }
  for (int i = 0; i < K; ++i) {
    mabd_joint_desc dj = ctx->joints[jorder[i]];
    if (ctx->any_frame) {
      to_principal(ctx, dj.body_a, dj.anchor_a);
      to_principal(ctx, dj.body_a, dj.axis_a);
      to_principal(ctx, dj.body_a, dj.ref_a);
      to_principal(ctx, dj.body_b, dj.anchor_b);
      to_principal(ctx, dj.body_b, dj.axis_b);
      to_principal(ctx, dj.body_b, dj.ref_b);
    }
    const auto &d = dj;
    jtype[i] = (int8_t)d.type;
    ja[i] = ctx->internal_of_body[d.body_a];
    jb[i] = d.body_b >= 0 ? ctx->internal_of_body[d.body_b] : -1;
    uint8_t f = 0;
    if (!ctx->bodies[d.body_a].fixed) f |= JF_A_FREE;
    if (d.body_b >= 0) {
      f |= JF_B_BODY;
      if (!ctx->bodies[d.body_b].fixed) f |= JF_B_FREE;
    }
    jfl[i] = f;
    double na = std::sqrt(d.axis_a[0] * d.axis_a[0] + d.axis_a[1] * d.axis_a[1] + d.axis_a[2] * d.axis_a[2]);
    double nb = std::sqrt(d.axis_b[0] * d.axis_b[0] + d.axis_b[1] * d.axis_b[1] + d.axis_b[2] * d.axis_b[2]);
    for (int a = 0; a < 3; ++a) {
      pa1[(size_t)a * K + i] = d.anchor_a[a];
      pb1[(size_t)a * K + i] = d.anchor_b[a];
      double uaa = na > 0 ? d.axis_a[a] / na : 0.0, ubb = nb > 0 ? d.axis_b[a] / nb : 0.0;
      ua[(size_t)a * K + i] = uaa;
      if (d.type == MABD_JOINT_UNIVERSAL) {
        // b's axis as the point difference l a2 (weight 0 on translation)
        pa2[(size_t)a * K + i] = 0.0;
        pb2[(size_t)a * K + i] = d.axis_len * ubb;
      } else {
        pa2[(size_t)a * K + i] = d.anchor_a[a] + d.axis_len * uaa;
        pb2[(size_t)a * K + i] = d.anchor_b[a] + d.axis_len * ubb;
      }
    }
    if (d.type == MABD_JOINT_PRISMATIC) {
      // the off-axis points p + l c (c: the unit reference directions)
      const double nca = std::sqrt(d.ref_a[0] * d.ref_a[0] + d.ref_a[1] * d.ref_a[1] + d.ref_a[2] * d.ref_a[2]);
      const double ncb = std::sqrt(d.ref_b[0] * d.ref_b[0] + d.ref_b[1] * d.ref_b[1] + d.ref_b[2] * d.ref_b[2]);
      for (int a = 0; a < 3; ++a) {
        pa3[(size_t)a * K + i] = d.anchor_a[a] + d.axis_len * (d.ref_a[a] / nca);
        pb3[(size_t)a * K + i] = d.anchor_b[a] + d.axis_len * (d.ref_b[a] / ncb);
      }
    }
  }
  // incidence over internal order, joints sorted by internal index
  std::vector<int32_t> ioff(M + 1, 0), ijoint;
  std::vector<int8_t> iside;
  {
    std::vector<std::vector<std::pair<int, int>>> lists(M);
    for (int i = 0; i < K; ++i) {
      if (jfl[i] & JF_A_FREE) lists[ja[i]].push_back({i, 0});
      if (jfl[i] & JF_B_FREE) lists[jb[i]].push_back({i, 1});
    }
    for (int j = 0; j < M; ++j) {
      std::sort(lists[j].begin(), lists[j].end());
      ioff[j + 1] = ioff[j] + (int)lists[j].size();
      for (auto &e : lists[j]) {
        ijoint.push_back(e.first);
        iside.push_back((int8_t)e.second);
      }
    }
  }
  // processing orders of the per-joint and per-body kernels (CHUNK_ORDER):
  // each run of CHUNK_ORDER entries stably partitioned by a type key; left
  // out (identity) when no run mixes keys
  std::vector<int32_t> jord, bord;
  {
    auto chunk_order = [](int n, const std::vector<int> &key, std::vector<int32_t> &out) {
      out.resize(n);
      bool moved = false;
      for (int c0 = 0; c0 < n; c0 += CHUNK_ORDER) {
        const int c1 = std::min(n, c0 + CHUNK_ORDER);
        for (int i = c0; i < c1; ++i) out[i] = i;
        std::stable_sort(out.begin() + c0, out.begin() + c1, [&](int a, int b) { return key[a] < key[b]; });
        for (int i = c0; i < c1 && !moved; ++i) moved = out[i] != i;
      }
      if (!moved) out.clear();
    };
    std::vector<int> jkey(K), bkey(M);
    for (int i = 0; i < K; ++i) jkey[i] = jtype[i];
    for (int j = 0; j < M; ++j) {
      // joint types in incidence order, base 5 (0: none), first four joints
      int kv = 0;
      for (int e = ioff[j], t = 0; e < ioff[j + 1] && t < 4; ++e, ++t) kv = kv * 5 + 1 + jtype[ijoint[e]];
      bkey[j] = kv;
    }
    chunk_order(K, jkey, jord);
    chunk_order(M, bkey, bord);
  }
  // chain: a joint's diagonal block collects one part from each of its free
  // bodies, the lower one along the path (slot 0) and the upper one (slot 1)
  std::vector<uint8_t> cfl(K, 0);
  std::vector<int8_t> islot(std::max<size_t>(ijoint.size(), 1), 0);
  const bool chainlike = solver == MABD_SOLVER_CHAIN || solver == MABD_SOLVER_LOOP;
  if (chainlike) {
    for (int j = 0; j < M; ++j) {
      const int n = ioff[j + 1] - ioff[j];
      for (int e = ioff[j]; e < ioff[j + 1]; ++e) {
        const int k = ijoint[e];
        int other = -1;
        if (iside[e] == 0 && (jfl[k] & JF_B_FREE)) other = jb[k];
        if (iside[e] == 1 && (jfl[k] & JF_A_FREE)) other = ja[k];
        const int slot = (other >= 0 && other < j) ? 1 : 0;
        islot[e] = (int8_t)slot;
        cfl[k] |= slot == 0 ? 1 : 2;
      }
      if (n == 2) cfl[ijoint[ioff[j]]] |= 4;
    }
  }

  // ---- device buffers
  bool ok = true;
  const int Mx = std::max(M, 1), Kx = std::max(K, 1);
  auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
  };
  DevBodies &B = ctx->B;
  B.M = M;
  B.q = dnew<double>(ctx, 12 * (size_t)Mx, ok);
  B.qd = dnew<double>(ctx, 12 * (size_t)Mx, ok);
  double *dsig = dnew<double>(ctx, 3 * (size_t)Mx, ok);
  double *dmass = dnew<double>(ctx, Mx, ok);
  double *dvmu = dnew<double>(ctx, Mx, ok);
  double *dvlam = dnew<double>(ctx, Mx, ok);
  double *dhinv = dnew<double>(ctx, HINV_N * (size_t)Mx, ok);
  uint8_t *dfixed = dnew<uint8_t>(ctx, Mx, ok);
  B.R = dnew<double>(ctx, 9 * (size_t)Mx, ok);
  B.ubar = dnew<double>(ctx, 12 * (size_t)Mx, ok);
  DevJoints &J = ctx->J;
  J.K = K;
  int8_t *djt = dnew<int8_t>(ctx, Kx, ok);
  int32_t *dja = dnew<int32_t>(ctx, Kx, ok);
  int32_t *djb = dnew<int32_t>(ctx, Kx, ok);
  uint8_t *djf = dnew<uint8_t>(ctx, Kx, ok);
  double *dpa1 = dnew<double>(ctx, 3 * (size_t)Kx, ok);
  double *dpb1 = dnew<double>(ctx, 3 * (size_t)Kx, ok);
  double *dpa2 = dnew<double>(ctx, 3 * (size_t)Kx, ok);
  double *dpb2 = dnew<double>(ctx, 3 * (size_t)Kx, ok);
  double *dua = dnew<double>(ctx, 3 * (size_t)Kx, ok);
  double *dpa3 = has_prism ? dnew<double>(ctx, 3 * (size_t)Kx, ok) : nullptr;
  double *dpb3 = has_prism ? dnew<double>(ctx, 3 * (size_t)Kx, ok) : nullptr;
  J.RH = dnew<double>(ctx, 9 * (size_t)Kx, ok);
  J.c = dnew<double>(ctx, 5 * (size_t)Kx, ok);
  J.b = dnew<double>(ctx, 5 * (size_t)Kx, ok);
  J.lambda = dnew<double>(ctx, 5 * (size_t)Kx, ok);
  J.qf = full_grad ? dnew<double>(ctx, 15 * (size_t)Kx, ok) : nullptr;
  const bool mixed = ctx->cfg.precision != MABD_FP64;
  const bool f32dual = ctx->cfg.precision == MABD_MIXED_FP32_DUAL;
  float *dhinvf = nullptr;
  float *dpf[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  const int npf = has_prism ? 6 : 4;
  if (mixed) {
    dhinvf = dnew<float>(ctx, HINV_N * (size_t)Mx, ok);
    B.fbh = dnew<float>(ctx, 12 * (size_t)Mx, ok);
    B.fbl = dnew<float>(ctx, 12 * (size_t)Mx, ok);
    B.Rlo = dnew<float>(ctx, 9 * (size_t)Mx, ok);
    B.dqb = dnew<double>(ctx, 12 * (size_t)Mx, ok);
    B.ubf = dnew<float>(ctx, 12 * (size_t)Mx, ok);
    B.Rf = dnew<float>(ctx, 9 * (size_t)Mx, ok);
    J.dlam = dnew<double>(ctx, 5 * (size_t)Kx, ok);
    J.RHf = dnew<float>(ctx, 9 * (size_t)Kx, ok);
    for (int i = 0; i < npf; ++i) dpf[i] = dnew<float>(ctx, 3 * (size_t)Kx, ok);
  }
  int32_t *djord = jord.empty() ? nullptr : dnew<int32_t>(ctx, jord.size(), ok);
  int32_t *dbord = bord.empty() ? nullptr : dnew<int32_t>(ctx, bord.size(), ok);
  int32_t *dioff = dnew<int32_t>(ctx, (size_t)M + 1, ok);
  int32_t *dij = dnew<int32_t>(ctx, std::max<size_t>(ijoint.size(), 1), ok);
  int8_t *dis = dnew<int8_t>(ctx, std::max<size_t>(iside.size(), 1), ok);
  ctx->d_status = dnew<int>(ctx, 1, ok);
  if (!ok) {
    free_all(ctx);
    return MABD_ERR_OUT_OF_MEMORY;
  }
  CK(up(B.q, q.data(), q.size() * 8));
  CK(up(B.qd, qd.data(), qd.size() * 8));
  CK(up(dsig, sig.data(), sig.size() * 8));
  CK(up(dmass, mass.data(), mass.size() * 8));
  CK(up(dvmu, vmu.data(), vmu.size() * 8));
  CK(up(dvlam, vlam.data(), vlam.size() * 8));
  CK(up(dhinv, hinv.data(), hinv.size() * 8));
  std::vector<float> hinvf;
  if (mixed) {
    hinvf.assign(hinv.begin(), hinv.end());
    CK(up(dhinvf, hinvf.data(), hinvf.size() * 4));
    CK(cudaMemsetAsync(B.dqb, 0, 12 * (size_t)Mx * 8, ctx->stream));
    CK(cudaMemsetAsync(J.dlam, 0, 5 * (size_t)Kx * 8, ctx->stream));
    CK(cudaMemsetAsync(J.RHf, 0, 9 * (size_t)Kx * 4, ctx->stream));
    const std::vector<double> *src[6] = {&pa1, &pb1, &pa2, &pb2, &pa3, &pb3};
    for (int i = 0; i < npf; ++i) {
      std::vector<float> f(src[i]->begin(), src[i]->end());
      CK(up(dpf[i], f.data(), f.size() * 4));
    }
    J.pa1f = dpf[0];
    J.pb1f = dpf[1];
    J.pa2f = dpf[2];
    J.pb2f = dpf[3];
    J.pa3f = dpf[4];
    J.pb3f = dpf[5];
  }
  CK(up(dfixed, fixed.data(), fixed.size()));
  CK(up(djt, jtype.data(), jtype.size()));
  CK(up(dja, ja.data(), ja.size() * 4));
  CK(up(djb, jb.data(), jb.size() * 4));
  CK(up(djf, jfl.data(), jfl.size()));
  CK(up(dpa1, pa1.data(), pa1.size() * 8));
  CK(up(dpb1, pb1.data(), pb1.size() * 8));
  CK(up(dpa2, pa2.data(), pa2.size() * 8));
  CK(up(dpb2, pb2.data(), pb2.size() * 8));
  CK(up(dua, ua.data(), ua.size() * 8));
  if (has_prism) {
    CK(up(dpa3, pa3.data(), pa3.size() * 8));
    CK(up(dpb3, pb3.data(), pb3.size() * 8));
  }
  if (djord) CK(up(djord, jord.data(), jord.size() * 4));
  if (dbord) CK(up(dbord, bord.data(), bord.size() * 4));
  J.order = djord;
  B.order = dbord;
  CK(up(dioff, ioff.data(), ioff.size() * 4));
  CK(up(dij, ijoint.data(), ijoint.size() * 4));
  CK(up(dis, iside.data(), iside.size()));
  CK(cudaMemsetAsync(J.lambda, 0, 5 * (size_t)Kx * 8, ctx->stream));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
  B.sig = dsig;
  B.mass = dmass;
  B.vmu = dvmu;
  B.vlam = dvlam;
  B.hinv = dhinv;
  B.hinvf = dhinvf;
  B.fixed = dfixed;
  J.type = djt;
  J.ja = dja;
  J.jb = djb;
  J.flags = djf;
  J.pa1 = dpa1;
  J.pb1 = dpb1;
  J.pa2 = dpa2;
  J.pb2 = dpb2;
  J.pa3 = dpa3;
  J.pb3 = dpb3;
  J.xj = pcg_only;
  J.ua = dua;
  ctx->I.off = dioff;
  ctx->I.joint = dij;
  ctx->I.side = dis;

  if (chainlike) {
    DevChain &C = ctx->C;
    C.K = K;
    C.Dfirst = dnew<double>(ctx, 15 * (size_t)K, ok);
    C.Dsecond = dnew<double>(ctx, 15 * (size_t)K, ok);
    C.B = dnew<double>(ctx, 25 * (size_t)K, ok);
    // a loop reduces the chain of its first K - 1 joints; the last joint is
    // the loop breaker (Sec. 5.4, Case III)
    const int Kr = solver == MABD_SOLVER_LOOP ? K - 1 : K;
    if (solver == MABD_SOLVER_LOOP) {
      C.corner = dnew<double>(ctx, 25, ok);
      ctx->loop_b = dnew<double>(ctx, 5 * (size_t)K, ok);
      ctx->loop_x = dnew<double>(ctx, 5 * (size_t)K, ok);
      ctx->loop_w = dnew<double>(ctx, 5 * 10, ok);
      ctx->loop_rows = jtype[K - 1] == 1 ? 5 : 3;
    }
    uint8_t *dcf = dnew<uint8_t>(ctx, K, ok);
    int8_t *dslot = dnew<int8_t>(ctx, islot.size(), ok);
    // Level-0 offset: with off = 1 a decoupled identity row precedes the first
    // joint, which shifts which rows level 0 eliminates.  The cheaper of the
    // two orders (FMA model of the reduction kernel) is used: for chains that
    // alternate balls and hinges it makes level 0 eliminate the hinges and
    // leaves only 3x3 rows above it.
    {
      std::vector<int> sz(Kr);
      for (int k = 0; k < Kr; ++k) sz[k] = jtype[k] == 1 ? 5 : 3;
      auto cost = [&](int off) {
        std::vector<int> cur(off, 3);
        cur.insert(cur.end(), sz.begin(), sz.end());
        double total = 0.0;
        while (cur.size() > 1) {
          const int N = (int)cur.size();
          std::vector<int> nxt;
          for (int n = 1; n < N; n += 2) {
            const double c = cur[n], l = cur[n - 1], r = n + 1 < N ? cur[n + 1] : 0;
            const double chol = c == 3 ? 7 : 30;
            total += chol + (l + r + 1) * c * (c + 1) / 2 + (l * (l + 1) / 2 + r * (r + 1) / 2 + l * r + l + r) * c;
          }
          for (int n = 0; n < N; n += 2) nxt.push_back(cur[n]);
          cur.swap(nxt);
        }
        return total;
      };
      C.off = (Kr > 1 && cost(1) < cost(0)) ? 1 : 0;
    }
    // cyclic-reduction levels
    ctx->levels.clear();
    int N = Kr + C.off;
    int lvl = 0;
    while (true) {
      CRLevel L{};
      L.N = N;
      if (lvl > 0) {
        L.D = dnew<double>(ctx, 15 * (size_t)N, ok);
        L.B = dnew<double>(ctx, 25 * (size_t)N, ok);
        L.b = dnew<double>(ctx, 5 * (size_t)N, ok);
        L.lam = dnew<double>(ctx, 5 * (size_t)N, ok);
      } else {
        L.lam = J.lambda;  // written through the offset by the back-substitution
      }
      if (N / 2 > 0) L.fac = dnew<double>(ctx, 70 * (size_t)(N / 2), ok);
      ctx->levels.push_back(L);
      if (N == 1) break;
      N = (N + 1) / 2;
      ++lvl;
    }
    if (f32dual) {
      ctx->levels_f.clear();
      for (size_t l = 0; l < ctx->levels.size(); ++l) {
        CRLevelT<float> Lf{};
        const int Nl = ctx->levels[l].N;
        Lf.N = Nl;
        if (l > 0) {
          Lf.D = dnew<float>(ctx, 15 * (size_t)Nl, ok);
          Lf.B = dnew<float>(ctx, 25 * (size_t)Nl, ok);
          Lf.b = dnew<float>(ctx, 5 * (size_t)Nl, ok);
          Lf.lam = dnew<float>(ctx, 5 * (size_t)Nl, ok);
        }
        if (Nl / 2 > 0) Lf.fac = dnew<float>(ctx, 70 * (size_t)(Nl / 2), ok);
        ctx->levels_f.push_back(Lf);
      }
      C.Dfirst_f = dnew<float>(ctx, 15 * (size_t)K, ok);
      C.Dsecond_f = dnew<float>(ctx, 15 * (size_t)K, ok);
      C.B_f = dnew<float>(ctx, 25 * (size_t)K, ok);
    }
    // The small levels run in one single-CTA launch per pass where a row's
    // serial latency is short (FP32 reduction): from the first level with at
    // most CR_TAIL_ROWS rows.  MABD_CR_TAIL=<rows> sets the bound for either
    // precision (0: off).
    {
      const int nl = (int)ctx->levels.size();
      int tail_rows = f32dual ? CR_TAIL_ROWS : 0;
      if (const char *e = std::getenv("MABD_CR_TAIL")) tail_rows = std::atoi(e);
      ctx->cr_tail_level = nl;
      if (tail_rows > 0)
        for (int l = 0; l < nl; ++l)
          if (ctx->levels[l].N <= tail_rows) {
            ctx->cr_tail_level = l;
            break;
          }
      ctx->d_levels = dnew<CRLevel>(ctx, nl, ok);
      if (ok) CK(cudaMemcpy(ctx->d_levels, ctx->levels.data(), nl * sizeof(CRLevel), cudaMemcpyHostToDevice));
      if (f32dual) {
        ctx->d_levels_f = dnew<CRLevelT<float>>(ctx, nl, ok);
        if (ok)
          CK(cudaMemcpy(ctx->d_levels_f, ctx->levels_f.data(), nl * sizeof(CRLevelT<float>),
                        cudaMemcpyHostToDevice));
      }
    }
    const size_t half = std::max((K + 1) / 2, 1);
    ctx->cL = dnew<double>(ctx, 20 * half, ok);
    ctx->cR = dnew<double>(ctx, 20 * half, ok);
    ctx->Bn = dnew<double>(ctx, 25 * half, ok);
    if (!ok) {
      free_all(ctx);
      return MABD_ERR_OUT_OF_MEMORY;
    }
    CK(up(dcf, cfl.data(), cfl.size()));
    CK(up(dslot, islot.data(), islot.size()));
    C.jflags = dcf;
    C.islot = dslot;
    if (ctx->loop_b) CK(cudaMemsetAsync(ctx->loop_b, 0, 5 * (size_t)K * 8, ctx->stream));
  }
  // segment-tiled chain step (k_seg.cu) for the FP32-reduction form with one
  // correction sweep, ball and hinge joints between chain bodies or to the
  // world (joints to fixed bodies keep the level-by-level reduction), when
  // MABD_CHAIN_SEG=1 (measured slower than the level-by-level reduction on
  // the 1M chain: the default stays the latter)
  ctx->seg_on = false;
  if (solver == MABD_SOLVER_CHAIN && f32dual && ctx->cfg.refine_steps == 1) {
    const char *e = std::getenv("MABD_CHAIN_SEG");
    bool want = e && e[0] == '1';
    int nb = 0;
    for (int j = 0; j < M; ++j) nb += fixed[j] ? 0 : 1;
    for (int k = 0; k < K && want; ++k)
      if (!(jfl[k] & JF_A_FREE) || ((jfl[k] & JF_B_BODY) && !(jfl[k] & JF_B_FREE))) want = false;
    // joint k joins path bodies k - 1 + sigma and k + sigma
    const int sigma = (K > 0 && jb[0] >= 0) ? 1 : 0;
    std::vector<uint8_t> cjf(K, 0);
    for (int k = 0; k < K && want; ++k) {
      const int lo = k - 1 + sigma, upb = k + sigma;
      uint8_t f = jtype[k] == 1 ? SEGJ_HINGE : 0;
      if (jb[k] >= 0) {
        if (ja[k] == lo && jb[k] == upb) f |= SEGJ_LO | SEGJ_UP | SEGJ_A_LO;
        else if (ja[k] == upb && jb[k] == lo) f |= SEGJ_LO | SEGJ_UP;
        else want = false;
      } else {
        if (ja[k] == lo) f |= SEGJ_LO | SEGJ_A_LO;
        else if (ja[k] == upb) f |= SEGJ_UP;
        else want = false;
      }
      if ((f & SEGJ_LO) && (lo < 0 || lo >= nb)) want = false;
      if ((f & SEGJ_UP) && (upb < 0 || upb >= nb)) want = false;
      cjf[k] = f;
    }
    // neighbouring joints share a body
    for (int k = 0; k + 1 < K && want; ++k)
      if (!(cjf[k] & SEGJ_UP) || !(cjf[k + 1] & SEGJ_LO)) want = false;
    if (want) {
      CK(seg_init());
      SegChain &S = ctx->seg;
      S.nb = nb;
      S.sigma = sigma;
      uint8_t *dcjf = dnew<uint8_t>(ctx, K, ok);
      S.ytile = dnew<float>(ctx, 5 * (size_t)K, ok);
      S.lam0 = dnew<float>(ctx, 5 * (size_t)K, ok);
      S.dq0 = dnew<float>(ctx, 12 * (size_t)nb, ok);
      S.z = dnew<float>(ctx, 12 * (size_t)nb, ok);
      S.u = dnew<float>(ctx, 12 * (size_t)nb, ok);
      S.rf = dnew<float>(ctx, 12 * (size_t)nb, ok);
      S.RHlo = dnew<float>(ctx, 9 * (size_t)K, ok);
      S.fac = dnew<float>(ctx, (size_t)65 * (SEG_T + 4) * ((K + SEG_T - 1) / SEG_T), ok);
      ctx->seg_lv.clear();
      int ut = SEG_UP_T;
      if (const char *u = std::getenv("MABD_SEG_UP_T")) {
        const int v = std::atoi(u);
        if (v >= 2 && v <= SEG_UP_T && (v & (v - 1)) == 0) ut = v;
      }
      ctx->seg_up_t = ut;
      int N = (K + SEG_T - 1) / SEG_T;
      while (true) {
        SegLevel L{};
        L.N = N;
        L.Dn = dnew<float>(ctx, 15 * (size_t)N, ok);
        L.Da = dnew<float>(ctx, 15 * (size_t)N, ok);
        L.Bn = dnew<float>(ctx, 25 * (size_t)N, ok);
        for (int ps = 0; ps < 2; ++ps) {
          L.r[ps].bn = dnew<float>(ctx, 5 * (size_t)N, ok);
          L.r[ps].ba = dnew<float>(ctx, 5 * (size_t)N, ok);
          L.r[ps].lam = dnew<float>(ctx, 5 * (size_t)N, ok);
          if (ctx->seg_lv.empty()) {
            L.r[ps].b0 = dnew<double>(ctx, 5 * (size_t)N, ok);
            L.r[ps].dl = dnew<double>(ctx, 5 * (size_t)N, ok);
          }
        }
        ctx->seg_lv.push_back(L);
        if (N <= ut) break;
        N = (N + ut - 1) / ut;
      }
      if (!ok) {
        free_all(ctx);
        return MABD_ERR_OUT_OF_MEMORY;
      }
      CK(up(dcjf, cjf.data(), cjf.size()));
      S.cjf = dcjf;
      ctx->seg_on = true;
    }
  }
  if (solver == MABD_SOLVER_PCG && mixed) {
    DevPCG32 &Q = ctx->P32;
    Q.nblocks = (K + 127) / 128;
    Q.r = dnew<float>(ctx, 5 * (size_t)Kx, ok);
    Q.z = dnew<float>(ctx, 5 * (size_t)Kx, ok);
    Q.p = dnew<float>(ctx, 5 * (size_t)Kx, ok);
    Q.Sp = dnew<float>(ctx, 5 * (size_t)Kx, ok);
    Q.x = dnew<float>(ctx, 5 * (size_t)Kx, ok);
    Q.zb = dnew<float>(ctx, 12 * (size_t)Mx, ok);
    Q.Lpre = dnew<float>(ctx, 15 * (size_t)Kx, ok);
    Q.part = dnew<double>(ctx, 2 * (size_t)std::max(Q.nblocks, 1), ok);
    Q.scal = dnew<double>(ctx, 8, ok);
    Q.iter = dnew<int>(ctx, 2, ok);
    Q.ppart = dnew<double>(ctx, 3 * (size_t)P32_MAXB, ok);
    Q.bar = dnew<unsigned>(ctx, 4, ok);
    if (!ok) {
      free_all(ctx);
      return MABD_ERR_OUT_OF_MEMORY;
    }
    if (!ctx->h_iter) {
      CK(cudaMallocHost((void **)&ctx->h_iter, 2 * sizeof(int)));
      CK(cudaMallocHost((void **)&ctx->h_scal, 8 * sizeof(double)));
    }
    // MABD_PCG_PERSIST=1: the persistent solve (one cooperative launch per
    // solve, the loop and its convergence test on the device) when the
    // device can run it.  Off by default: on the 64x64x16 net it measured
    // 63.4 ms per step against 57.9 ms for one launch per step of an
    // iteration (both ~0.1 ms per iteration, bound by the gathers' memory
    // latency; the persistent form adds five grid barriers per iteration).
    const char *pe = std::getenv("MABD_PCG_PERSIST");
    int coop = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (coop && pe && pe[0] == '1') {
      ctx->p32_nb[0] = p32_persist_blocks(ctx->J.xj, false);
      ctx->p32_nb[1] = p32_persist_blocks(ctx->J.xj, true);
    }
  }
  if (solver == MABD_SOLVER_PCG && !mixed) {
    DevPCG &P = ctx->P;
    P.nblocks = (K + 127) / 128;
    P.r = dnew<double>(ctx, 5 * (size_t)Kx, ok);
    P.z = dnew<double>(ctx, 5 * (size_t)Kx, ok);
    P.p = dnew<double>(ctx, 5 * (size_t)Kx, ok);
    P.Sp = dnew<double>(ctx, 5 * (size_t)Kx, ok);
    P.zb = dnew<double>(ctx, 12 * (size_t)Mx, ok);
    P.Lpre = dnew<double>(ctx, 15 * (size_t)Kx, ok);
    P.part = dnew<double>(ctx, 2 * (size_t)std::max(P.nblocks, 1), ok);
    P.scal = dnew<double>(ctx, 8, ok);
    P.iter = dnew<int>(ctx, 2, ok);
    if (!ok) {
      free_all(ctx);
      return MABD_ERR_OUT_OF_MEMORY;
    }
    if (!ctx->h_iter) {
      CK(cudaMallocHost((void **)&ctx->h_iter, 2 * sizeof(int)));
      CK(cudaMallocHost((void **)&ctx->h_scal, 8 * sizeof(double)));
    }
  }
  if (solver == MABD_SOLVER_TREE) {
    DevTree &T = ctx->T;
    const int nr = std::max(tord.nroots, 1);
    std::vector<int32_t> rj(2 * (size_t)nr, -1);
    for (int i = 0; i < 2 * tord.nroots; ++i)
      rj[i] = tord.root_joint[i] >= 0 ? ctx->internal_of_joint[tord.root_joint[i]] : -1;
    T.nroots = tord.nroots;
    int32_t *dpar = dnew<int32_t>(ctx, Mx, ok);
    int32_t *dpj = dnew<int32_t>(ctx, Mx, ok);
    int8_t *dps = dnew<int8_t>(ctx, Mx, ok);
    int32_t *dcf = dnew<int32_t>(ctx, Mx, ok);
    int32_t *dcc = dnew<int32_t>(ctx, Mx, ok);
    int32_t *drid = dnew<int32_t>(ctx, Mx, ok);
    int32_t *drj = dnew<int32_t>(ctx, rj.size(), ok);
    int8_t *drs = dnew<int8_t>(ctx, tord.root_side.size(), ok);
    T.X = dnew<double>(ctx, 60 * (size_t)Mx, ok);
    T.LD = dnew<double>(ctx, 15 * (size_t)Mx, ok);
    T.y = dnew<double>(ctx, 12 * (size_t)Mx, ok);
    T.e = dnew<double>(ctx, 5 * (size_t)Mx, ok);
    T.U = dnew<double>(ctx, 60 * (size_t)Mx, ok);
    T.v = dnew<double>(ctx, 12 * (size_t)Mx, ok);
    T.dq = dnew<double>(ctx, 12 * (size_t)Mx, ok);
    T.rX = dnew<double>(ctx, 120 * (size_t)nr, ok);
    T.rLD = dnew<double>(ctx, 55 * (size_t)nr, ok);
    T.re = dnew<double>(ctx, 10 * (size_t)nr, ok);
    // the FP64 form's solve: C(q_n) weighted by residual_rhs, multipliers to
    // J.lambda, the state updated by the downward pass
    T.c = J.c;
    T.crr = ctx->cfg.residual_rhs ? 1.0 : 0.0;
    T.lam = J.lambda;
    T.lam_acc = nullptr;
    T.dqb = nullptr;
    T.dqb_add = 0;
    if (f32dual) {
      DevTreeT<float> &Tf = ctx->Tf;
      Tf.X = dnew<float>(ctx, 60 * (size_t)Mx, ok);
      Tf.LD = dnew<float>(ctx, 15 * (size_t)Mx, ok);
      Tf.y = dnew<float>(ctx, 12 * (size_t)Mx, ok);
      Tf.e = dnew<float>(ctx, 5 * (size_t)Mx, ok);
      Tf.U = dnew<float>(ctx, 60 * (size_t)Mx, ok);
      Tf.v = dnew<float>(ctx, 12 * (size_t)Mx, ok);
      Tf.dq = dnew<float>(ctx, 12 * (size_t)Mx, ok);
      Tf.rX = dnew<float>(ctx, 120 * (size_t)nr, ok);
      Tf.rLD = dnew<float>(ctx, 55 * (size_t)nr, ok);
      Tf.re = dnew<float>(ctx, 10 * (size_t)nr, ok);
      // the first solve of a step; the correction solves set their own
      Tf.c = J.c;
      Tf.crr = T.crr;
      Tf.lam = J.lambda;
      Tf.lam_acc = nullptr;
      Tf.dqb = B.dqb;
      Tf.dqb_add = 0;
    }
    if (!ok) {
      free_all(ctx);
      return MABD_ERR_OUT_OF_MEMORY;
    }
    std::vector<int32_t> tpj(M, -1);
    for (int i = 0; i < M; ++i)
      if (tord.parent[i] >= 0) tpj[i] = ctx->internal_of_joint[tord.pjoint[i]];
    CK(up(dpar, tord.parent.data(), (size_t)M * 4));
    CK(up(dpj, tpj.data(), (size_t)M * 4));
    CK(up(dps, tord.pside.data(), (size_t)M));
    CK(up(dcf, tord.cfirst.data(), (size_t)M * 4));
    CK(up(dcc, tord.ccount.data(), (size_t)M * 4));
    CK(up(drid, tord.root_id.data(), (size_t)M * 4));
    CK(up(drj, rj.data(), rj.size() * 4));
    CK(up(drs, tord.root_side.data(), tord.root_side.size()));
    T.parent = dpar;
    T.pjoint = dpj;
    T.pside = dps;
    T.cfirst = dcf;
    T.ccount = dcc;
    T.root_id = drid;
    T.root_joint = drj;
    T.root_side = drs;
    ctx->tree_lvl = tord.lvl_off;
    // per level, the bodies with children first, then the leaves (index
    // lists, so that each upward kernel runs uniform warps while siblings
    // stay contiguous in the body order)
    std::vector<int32_t> ids;
    ctx->tree_mid.assign(tord.lvl_off.size(), 0);
    for (size_t l = 0; l + 1 < tord.lvl_off.size(); ++l) {
      for (int i = tord.lvl_off[l]; i < tord.lvl_off[l + 1]; ++i)
        if (tord.ccount[i] > 0) ids.push_back(i);
      ctx->tree_mid[l] = (int32_t)ids.size();
      for (int i = tord.lvl_off[l]; i < tord.lvl_off[l + 1]; ++i)
        if (tord.ccount[i] == 0) ids.push_back(i);
    }
    // narrow levels (at most MABD_TREE_NARROW bodies, default 256; 0: none)
    // run their downward pass together in one block
    {
      int nn = 256;
      if (const char *e = std::getenv("MABD_TREE_NARROW")) nn = std::max(0, std::atoi(e));
      const int nlev = (int)tord.lvl_off.size() - 1;
      ctx->tree_narrow.assign(std::max(nlev, 0), 0);
      for (int l = 0; l < nlev; ++l) ctx->tree_narrow[l] = tord.lvl_off[l + 1] - tord.lvl_off[l] <= nn;
    }
    int32_t *dids = dnew<int32_t>(ctx, std::max<size_t>(ids.size(), 1), ok);
    int32_t *dlo = dnew<int32_t>(ctx, tord.lvl_off.size(), ok);
    if (!ok) {
      free_all(ctx);
      return MABD_ERR_OUT_OF_MEMORY;
    }
    CK(up(dids, ids.data(), ids.size() * 4));
    CK(up(dlo, tord.lvl_off.data(), tord.lvl_off.size() * 4));
    ctx->T.order = dids;
    ctx->T.lv_lo = dlo;
    if (f32dual) {
      DevTreeT<float> &Tf = ctx->Tf;
      Tf.parent = T.parent;
      Tf.pjoint = T.pjoint;
      Tf.pside = T.pside;
      Tf.cfirst = T.cfirst;
      Tf.ccount = T.ccount;
      Tf.root_id = T.root_id;
      Tf.root_joint = T.root_joint;
      Tf.root_side = T.root_side;
      Tf.nroots = T.nroots;
      Tf.order = dids;
      Tf.lv_lo = dlo;
    }
    // the same bodies tree by tree: per tree and depth, bodies with children
    // first, then leaves; a sentinel record closes each tree
    {
      const int nlev = (int)tord.lvl_off.size() - 1;
      const int ntrees = nlev > 0 ? tord.lvl_off[1] - tord.lvl_off[0] : 0;
      std::vector<int32_t> root_of(M, -1), depth(M, 0);
      for (int l = 0; l < nlev; ++l)
        for (int i = tord.lvl_off[l]; i < tord.lvl_off[l + 1]; ++i) {
          depth[i] = l;
          root_of[i] = tord.parent[i] < 0 ? i : root_of[tord.parent[i]];
        }
      std::vector<std::vector<std::vector<int32_t>>> bucket(ntrees);
      for (int l = 0; l < nlev; ++l)
        for (int i = tord.lvl_off[l]; i < tord.lvl_off[l + 1]; ++i) {
          auto &bt = bucket[root_of[i] - tord.lvl_off[0]];
          if ((int)bt.size() <= l) bt.resize(l + 1);
          bt[l].push_back(i);
        }
      // deepest trees first (then the larger): the persistent kernel's blocks
      // take trees in this order, so the longest dependent chains start first
      std::vector<int32_t> tsz(ntrees, 0), torder(ntrees);
      for (int t = 0; t < ntrees; ++t) {
        for (auto &lvl : bucket[t]) tsz[t] += (int32_t)lvl.size();
        torder[t] = t;
      }
      std::stable_sort(torder.begin(), torder.end(), [&](int32_t a, int32_t b) {
        if (bucket[a].size() != bucket[b].size()) return bucket[a].size() > bucket[b].size();
        return tsz[a] > tsz[b];
      });
      std::vector<int32_t> tlvl(std::max(ntrees, 1)), tnl(std::max(ntrees, 1)), flo, fmid, ford;
      for (int t = 0; t < ntrees; ++t) {
        tlvl[t] = (int32_t)flo.size();
        tnl[t] = (int32_t)bucket[torder[t]].size();
        for (auto &lvl : bucket[torder[t]]) {
          flo.push_back((int32_t)ford.size());
          for (int i : lvl)
            if (tord.ccount[i] > 0) ford.push_back(i);
          fmid.push_back((int32_t)ford.size());
          for (int i : lvl)
            if (tord.ccount[i] == 0) ford.push_back(i);
        }
        flo.push_back((int32_t)ford.size());
        fmid.push_back((int32_t)ford.size());
      }
      int32_t *d1 = dnew<int32_t>(ctx, tlvl.size(), ok), *d2 = dnew<int32_t>(ctx, tnl.size(), ok);
      int32_t *d3 = dnew<int32_t>(ctx, std::max<size_t>(flo.size(), 1), ok);
      int32_t *d4 = dnew<int32_t>(ctx, std::max<size_t>(fmid.size(), 1), ok);
      int32_t *d5 = dnew<int32_t>(ctx, std::max<size_t>(ford.size(), 1), ok);
      if (!ok) {
        free_all(ctx);
        return MABD_ERR_OUT_OF_MEMORY;
      }
      CK(up(d1, tlvl.data(), tlvl.size() * 4));
      CK(up(d2, tnl.data(), tnl.size() * 4));
      CK(up(d3, flo.data(), flo.size() * 4));
      CK(up(d4, fmid.data(), fmid.size() * 4));
      CK(up(d5, ford.data(), ford.size() * 4));
      DevForest &F = ctx->F;
      F.ntrees = ntrees;
      F.tlvl = d1;
      F.tnl = d2;
      F.lo = d3;
      F.mid = d4;
      F.order = d5;
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->sp.h = h;
  ctx->sp.inv_h = 1.0 / h;
  for (int a = 0; a < 3; ++a) ctx->sp.g[a] = ctx->cfg.gravity[a];
  ctx->sp.residual_rhs = ctx->cfg.residual_rhs ? 1 : 0;
  ctx->sp.rot_norm = ctx->cfg.rotation_mode == MABD_ROTATION_NORMALIZED ? 1 : 0;
  if (solver == MABD_SOLVER_TREE && K > 0) {
    mabd_status st = tune_tree(ctx);
    if (st) return st;
  }
  ctx->frozen = true;
  return MABD_OK;
}

// One step is enqueued in three phases so that it can be captured into CUDA
// graphs: `pre` runs everything up to the dual solve (the whole solve for
// chains and trees, the set-up for PCG), the PCG iterations run in chunks,
// and `post` back-propagates (and, with statistics, computes residuals).
// cyclic reduction of the chain's dual: factorization of the current blocks
// with the current rhs, or (rhs_only) a new rhs J.b through the stored
// factors; level 0 writes its solution to Jout.lambda and adds it to acc
}  // extern "C"

template <typename T>
static void enqueue_cr_t(mabd_ctx *ctx, cudaStream_t s, bool rhs_only, const DevJoints &Jin,
                         const DevJoints &Jout, double *acc, std::vector<CRLevelT<T>> &levels,
                         const CRLevelT<T> *d_levels) {
  const int nl = (int)levels.size();
  const int l0 = ctx->cr_tail_level;
  if (l0 < nl) {
    // large levels one launch each, the rest in the single-CTA tail
    for (int l = 0; l < l0; ++l) {
      if (rhs_only)
        run(ctx, "cr_rhs", [&] { launch_cr_rhs<T>(ctx->C, Jin, levels[l], l, levels[l + 1], s); });
      else
        run(ctx, "cr_level",
            [&] { launch_cr_level<T>(ctx->C, Jin, levels[l], l, levels[l + 1], ctx->d_status, s); });
    }
    run(ctx, "cr_tail", [&] {
      launch_cr_tail<T>(ctx->C, Jin, Jout, d_levels, l0, nl, rhs_only, (T *)ctx->cL, (T *)ctx->cR,
                        (T *)ctx->Bn, ctx->d_status, l0 == 0 ? acc : nullptr, s);
    });
    for (int l = l0 - 1; l >= 0; --l)
      run(ctx, "cr_back", [&] {
        launch_cr_back<T>(ctx->C, l == 0 ? Jout : Jin, levels[l], levels[l + 1], l, s, l == 0 ? acc : nullptr);
      });
    return;
  }
  for (int l = 0; l + 1 < nl; ++l) {
    if (rhs_only)
      run(ctx, "cr_rhs", [&] { launch_cr_rhs<T>(ctx->C, Jin, levels[l], l, levels[l + 1], s); });
    else
      run(ctx, "cr_level", [&] { launch_cr_level<T>(ctx->C, Jin, levels[l], l, levels[l + 1], ctx->d_status, s); });
  }
  if (nl == 1) {
    // a single row (one joint): level 0 is the top row, written to Jout.lambda
    run(ctx, "cr_top", [&] { launch_cr_top<T>(ctx->C, Jin, levels[0], 0, ctx->d_status, s, Jout.lambda, acc); });
    return;
  }
  run(ctx, "cr_top", [&] { launch_cr_top<T>(ctx->C, Jin, levels[nl - 1], nl - 1, ctx->d_status, s); });
  for (int l = nl - 2; l >= 0; --l)
    run(ctx, "cr_back", [&] {
      launch_cr_back<T>(ctx->C, l == 0 ? Jout : Jin, levels[l], levels[l + 1], l, s, l == 0 ? acc : nullptr);
    });
}

// the chain's reduction in the precision of the form in use; the rhs comes
// from Jin.b (level 0), the solution goes to Jout.lambda (and acc)
static void enqueue_cr(mabd_ctx *ctx, cudaStream_t s, bool rhs_only, const DevJoints &Jout, double *acc,
                       const DevJoints *Jin = nullptr) {
  const DevJoints &Ji = Jin ? *Jin : ctx->J;
  if (ctx->cfg.precision == MABD_MIXED_FP32_DUAL)
    enqueue_cr_t<float>(ctx, s, rhs_only, Ji, Jout, acc, ctx->levels_f, ctx->d_levels_f);
  else
    enqueue_cr_t<double>(ctx, s, rhs_only, Ji, Jout, acc, ctx->levels, ctx->d_levels);
}

// Loop solver (k_loop.cu; Sec. 5.4, Case III): factor the chain of joints
// 0..K-2 with its rhs, one rhs pass per row of the breaker K-1 for
// S_cc^{-1} S_cl, the breaker's Schur complement, then a last rhs pass with
// b_c - S_cl lambda_L for the chain's multipliers
static void enqueue_loop(mabd_ctx *ctx, cudaStream_t s) {
  const int K = ctx->J.K;
  enqueue_cr(ctx, s, false, ctx->J, nullptr);
  DevJoints Jin = ctx->J, Jx = ctx->J;
  Jin.b = ctx->loop_b;
  Jx.lambda = ctx->loop_x;
  const int n = ctx->loop_rows;
  for (int t = 0; t < n; ++t) {
    run(ctx, "loop_schur", [&] { launch_loop_column(ctx->C, K, ctx->loop_b, t, s); });
    enqueue_cr(ctx, s, true, Jx, nullptr, &Jin);
    run(ctx, "loop_schur", [&] { launch_loop_gather(K, ctx->loop_x, ctx->loop_w, t, s); });
  }
  run(ctx, "loop_schur", [&] { launch_loop_schur(ctx->C, ctx->J, ctx->loop_w, ctx->d_status, s); });
  enqueue_cr(ctx, s, true, ctx->J, nullptr);
}

extern "C" {

// the upper systems of the segment-tiled chain step for one pass: reduce
// every level into the next, solve the last in one CTA, back-substitute down
static void enqueue_seg_up(mabd_ctx *ctx, int pass, unsigned long long *rmax, cudaStream_t s) {
  const int n = (int)ctx->seg_lv.size(), T = ctx->seg_up_t;
  for (int i = 0; i + 1 < n; ++i)
    run(ctx, "seg_up", [&] {
      launch_seg_up_reduce(ctx->seg_lv[i], ctx->seg_lv[i + 1], T, pass, pass == 0, i == 0 ? rmax : nullptr,
                           ctx->d_status, s);
    });
  run(ctx, "seg_up", [&] {
    launch_seg_up_top(ctx->seg_lv[n - 1], T, pass, n == 1 ? rmax : nullptr, ctx->d_status, s);
  });
  for (int i = n - 2; i >= 0; --i)
    run(ctx, "seg_up", [&] { launch_seg_up_back(ctx->seg_lv[i], ctx->seg_lv[i + 1], T, pass, ctx->d_status, s); });
}

// segment-tiled chain step (k_seg.cu): the approximate solve, the
// back-substitution with the residuals and the correction's rhs, the
// correction's back-substitution with the state update; each tile pass
// followed by the solve of the tiles' first rows
static void enqueue_seg_chain(mabd_ctx *ctx, unsigned long long *maxbits, cudaStream_t s) {
  SegChain S = ctx->seg;
  S.lv0 = ctx->seg_lv[0];
  S.write_cj = maxbits ? 1 : 0;
  S.refine_max = maxbits ? maxbits + 2 : nullptr;
  S.polar_iters = maxbits ? maxbits + 3 : nullptr;
  const StepParams &p = ctx->sp;
  run(ctx, "seg_body", [&] { launch_seg_body(ctx->B, ctx->J, p, S, ctx->d_status, s); });
  run(ctx, "seg_first", [&] { launch_seg_tiles(SEG_FIRST, ctx->B, ctx->J, p, S, ctx->d_status, s); });
  enqueue_seg_up(ctx, 0, nullptr, s);
  run(ctx, "seg_corr", [&] { launch_seg_tiles(SEG_CORR, ctx->B, ctx->J, p, S, ctx->d_status, s); });
  enqueue_seg_up(ctx, 1, S.refine_max, s);
  run(ctx, "seg_final", [&] { launch_seg_tiles(SEG_FINAL, ctx->B, ctx->J, p, S, ctx->d_status, s); });
}

// mixed-precision chain step (k_mixed.cu): approximate solve with FP32
// products and the FP64 reduction, then refine_steps FP64 residual-correction
// sweeps through the stored factors, then the state update
static void enqueue_mixed_chain(mabd_ctx *ctx, unsigned long long *maxbits, cudaStream_t s) {
  const StepParams &p = ctx->sp;
  if (ctx->seg_on) {
    enqueue_seg_chain(ctx, maxbits, s);
    return;
  }
  run(ctx, "mx_body_prep", [&] {
    launch_mx_body_prep(ctx->B, p, ctx->d_status, s, maxbits ? maxbits + 3 : nullptr);
  });
  if (ctx->J.K == 0) {
    run(ctx, "mx_final", [&] { launch_mx_final(ctx->B, ctx->J, ctx->I, p, MX_FROM_U, s); });
    return;
  }
  run(ctx, "mx_joint_prep", [&] { launch_mx_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s); });
  run(ctx, "mx_chain_gram", [&] {
    launch_mx_chain_gram(ctx->B, ctx->J, ctx->I, ctx->C, s, ctx->cfg.precision == MABD_MIXED_FP32_DUAL);
  });
  enqueue_cr(ctx, s, false, ctx->J, nullptr);
  const int sweeps = ctx->cfg.refine_steps;
  DevJoints Jc = ctx->J;
  Jc.lambda = ctx->J.dlam;
  for (int it = 0; it < sweeps; ++it) {
    run(ctx, "mx_res_body", [&] {
      launch_mx_res_body(ctx->B, ctx->J, ctx->I, p, it == 0 ? MX_FROM_U : MX_FROM_CORRECTION, s);
    });
    unsigned long long *mb = (maxbits && it == sweeps - 1) ? maxbits + 2 : nullptr;
    run(ctx, "mx_res_joint", [&] { launch_mx_res_joint(ctx->B, ctx->J, p, mb, s); });
    enqueue_cr(ctx, s, true, Jc, ctx->J.lambda);
  }
  run(ctx, "mx_final", [&] {
    launch_mx_final(ctx->B, ctx->J, ctx->I, p, sweeps == 0 ? MX_FROM_U : MX_FROM_CORRECTION, s);
  });
}

}  // extern "C"

// One solve of the KKT system by the tree elimination with T's right-hand
// side and outputs: the upward levels (deepest first, the tuned variant per
// level), then the downward levels, or the persistent kernel when the tuner
// chose it.
template <typename S>
static void enqueue_tree_solve(mabd_ctx *ctx, const DevTreeT<S> &T, cudaStream_t s) {
  const StepParams &p = ctx->sp;
  if (ctx->tree_mode != 0) {
    run(ctx, "tree_forest", [&] {
      launch_tree_forest(ctx->B, ctx->J, T, ctx->F, p, ctx->d_status, s, ctx->tree_mode);
    });
    return;
  }
  tree_levels(ctx, T, s, [&](const char *name, auto &&f) { run(ctx, name, f); });
}

extern "C" {

// Mixed-precision tree step (MABD_MIXED_FP32_DUAL): FP64 polar, rhs and
// constraint values; the tree elimination in FP32 gives lambda and the
// rest-frame increment dqb; each sweep forms the FP64 residuals (primal
// r = fbar - Hbar dqb - g(lambda) with z = Hbar^{-1} r, dual C + G dqb) and
// solves the correction system by the same FP32 elimination with z and
// C + G dqb as its right-hand side, adding to lambda and dqb; then the state
// update.
static void enqueue_mixed_tree(mabd_ctx *ctx, unsigned long long *maxbits, cudaStream_t s) {
  const StepParams &p = ctx->sp;
  run(ctx, "mx_body_prep", [&] {
    launch_mx_body_prep(ctx->B, p, ctx->d_status, s, maxbits ? maxbits + 3 : nullptr);
  });
  run(ctx, "mx_joint_prep", [&] { launch_mx_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s); });
  enqueue_tree_solve(ctx, ctx->Tf, s);
  DevTreeT<float> Tc = ctx->Tf;
  Tc.c = ctx->J.b;
  Tc.crr = 1.0;
  Tc.lam = ctx->J.dlam;
  Tc.lam_acc = ctx->J.lambda;
  Tc.dqb_add = 1;
  const int sweeps = ctx->cfg.refine_steps;
  for (int it = 0; it < sweeps; ++it) {
    run(ctx, "mx_res_body", [&] { launch_mx_res_body(ctx->B, ctx->J, ctx->I, p, MX_FROM_DQB, s); });
    unsigned long long *mb = (maxbits && it == sweeps - 1) ? maxbits + 2 : nullptr;
    run(ctx, "mx_res_joint", [&] { launch_mx_res_joint(ctx->B, ctx->J, p, mb, s, false); });
    enqueue_tree_solve(ctx, Tc, s);
  }
  run(ctx, "mx_final", [&] { launch_mx_final(ctx->B, ctx->J, ctx->I, p, MX_FROM_DQB, s); });
}

// iters (may be null): the step's polar-iteration counter
static void enqueue_pre(mabd_ctx *ctx, cudaStream_t s, unsigned long long *iters = nullptr) {
  const StepParams &p = ctx->sp;
  if (ctx->cfg.precision != MABD_FP64) return;  // the whole step is in enqueue_post
  run(ctx, "body_prep", [&] { launch_body_prep(ctx->B, p, ctx->d_status, s, iters); });
  if (ctx->J.K == 0) return;
  run(ctx, "joint_prep", [&] { launch_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s); });
  if (ctx->solver == MABD_SOLVER_CHAIN) {
    run(ctx, "chain_gram", [&] { launch_chain_gram(ctx->B, ctx->J, ctx->I, ctx->C, s); });
    enqueue_cr(ctx, s, false, ctx->J, nullptr);
  } else if (ctx->solver == MABD_SOLVER_LOOP) {
    run(ctx, "chain_gram", [&] { launch_chain_gram(ctx->B, ctx->J, ctx->I, ctx->C, s); });
    enqueue_loop(ctx, s);
  } else if (ctx->solver == MABD_SOLVER_TREE) {
    enqueue_tree_solve(ctx, ctx->T, s);
  } else if (ctx->solver == MABD_SOLVER_PCG) {
    run(ctx, "pcg_setup", [&] { launch_pcg_setup(ctx->B, ctx->J, ctx->P, ctx->cfg.pcg_rtol, ctx->d_status, s); });
  }
}

constexpr int PCG_CHUNK = 16;

static void enqueue_pcg_chunk(mabd_ctx *ctx, cudaStream_t s) {
  for (int i = 0; i < PCG_CHUNK; ++i)
    run(ctx, "pcg_iteration", [&] {
      launch_pcg_iteration(ctx->B, ctx->J, ctx->I, ctx->P, ctx->cfg.pcg_max_iters, s);
    });
}

static void enqueue_post(mabd_ctx *ctx, unsigned long long *maxbits, cudaStream_t s) {
  const StepParams &p = ctx->sp;
  if (ctx->cfg.precision != MABD_FP64 && ctx->J.K > 0 && ctx->solver == MABD_SOLVER_TREE)
    enqueue_mixed_tree(ctx, maxbits, s);
  else if (ctx->cfg.precision != MABD_FP64)
    enqueue_mixed_chain(ctx, maxbits, s);
  else if (!(ctx->J.K > 0 && ctx->solver == MABD_SOLVER_TREE))
    run(ctx, "backprop", [&] { launch_backprop(ctx->B, ctx->J, ctx->I, p, ctx->d_status, s); });
  if (maxbits && ctx->J.K > 0)
    run(ctx, "residuals", [&] { launch_residuals(ctx->B, ctx->J, p, maxbits, ctx->d_status, s); });
}

// Block-Jacobi PCG on the dual.  Iterations are enqueued in chunks of 16
// (replayed from a CUDA graph when graphs are on); between chunks the host
// reads the device's iteration count and convergence flag (the kernels of a
// converged iteration return immediately), so the loop is bounded by
// pcg_max_iters and nothing on the device waits.
static mabd_status pcg_loop(mabd_ctx *ctx, cudaStream_t s, cudaGraphExec_t chunk_graph) {
  const int max_it = ctx->cfg.pcg_max_iters;
  int done = 0;
  for (int launched = 0; launched < max_it && !done; launched += PCG_CHUNK) {
    if (chunk_graph) CK(cudaGraphLaunch(chunk_graph, s));
    else enqueue_pcg_chunk(ctx, s);
    CK(cudaMemcpyAsync(ctx->h_iter, ctx->P.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    done = ctx->h_iter[1];
  }
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->P.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_iter, ctx->P.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->pcg_last_iters = ctx->h_iter[0];
  const double bb = ctx->h_scal[4], rr = ctx->h_scal[3];
  ctx->pcg_last_rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  if (!(rr <= ctx->h_scal[5] * bb)) {
    int bits = ST_PCG_NOCONV;
    CK(cudaMemcpyAsync(&bits, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bits |= ST_PCG_NOCONV;
    CK(cudaMemcpyAsync(ctx->d_status, &bits, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return cuda_fail(ctx, cudaGetLastError());
}

// FP32 PCG solve of S x = rhs from x = 0 (mixed form, graphs); x goes to out,
// acc += x when acc is given.  Iterations are enqueued in chunks with a host
// check of the device's convergence flag between chunks, as for FP64 PCG.
constexpr double MIXED_INNER_RTOL = 1e-6;

static mabd_status p32_solve(mabd_ctx *ctx, cudaStream_t s, const double *rhs, double *out, double *acc,
                             bool learned);

// one FP32 PCG solve with the learned preconditioner when it is on; a learned
// solve that does not reach the tolerance within pcg_max_iters is repeated
// with block Jacobi (the fallback), which is then the solve that counts
static mabd_status p32_solve_any(mabd_ctx *ctx, cudaStream_t s, const double *rhs, double *out,
                                 double *acc) {
  if (!ctx->lpc_on) return p32_solve(ctx, s, rhs, out, acc, false);
  mabd_status st = p32_solve(ctx, s, rhs, out, nullptr, true);
  if (st) return st;
  const double bb = ctx->h_scal[4], rr = ctx->h_scal[3], tol2 = ctx->h_scal[5];
  if (std::isfinite(rr) && rr <= tol2 * bb) {
    if (acc) run(ctx, "p32_finish", [&] { launch_p32_finish(ctx->J, ctx->P32, out, acc, s); });
    return MABD_OK;
  }
  ++ctx->lpc_fallbacks;
  return p32_solve(ctx, s, rhs, out, acc, false);
}

static mabd_status p32_solve(mabd_ctx *ctx, cudaStream_t s, const double *rhs, double *out, double *acc,
                             bool learned) {
  const double rtol = std::max(ctx->cfg.pcg_rtol, MIXED_INNER_RTOL);
  DevPCG32 P = ctx->P32;
  if (!learned) P.t = nullptr;
  const LpcGraph *lg = learned ? &ctx->lg : nullptr;
  const LpcAct *la = learned ? &ctx->la : nullptr;
  const int max_it = ctx->cfg.pcg_max_iters;
  // ball-joint graphs whose C and E are current (learned preconditioner on):
  // the normalized-space solve
  const int nbn = ctx->lpc_on ? ctx->pn_nb[learned ? 1 : 0] : 0;
  if (nbn > 0) {
    // the step's first solve (of S lambda = b) starts from the multipliers
    // of the previous step (zero before the first); MABD_PCG_WARM=0: from 0
    const char *we = std::getenv("MABD_PCG_WARM");
    const bool warm = out == ctx->J.lambda && !acc && !(we && we[0] == '0');
    cudaError_t e = cudaSuccess;
    run(ctx, "p32_solve", [&] {
      e = launch_pcgn(ctx->lg, ctx->la, ctx->pn, ctx->P32, learned, rhs, warm ? ctx->J.lambda : nullptr, rtol, max_it,
                      out,
                      learned ? nullptr : acc, ctx->d_status, nbn, s);
    });
    CK(e);
    CK(cudaMemcpyAsync(ctx->h_scal, ctx->P32.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_iter, ctx->P32.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->pcg_last_iters += ctx->h_iter[0];
    const double bb = ctx->h_scal[4], rr = ctx->h_scal[3];
    ctx->pcg_last_rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    return MABD_OK;
  }
  const int nb = ctx->p32_nb[learned ? 1 : 0];
  if (nb > 0) {
    cudaError_t e = cudaSuccess;
    run(ctx, "p32_solve", [&] {
      e = launch_p32_persist(ctx->B, ctx->J, ctx->I, P, lg, la, rhs, rtol, max_it, out, learned ? nullptr : acc,
                             ctx->d_status, nb, s);
    });
    CK(e);
    CK(cudaMemcpyAsync(ctx->h_scal, ctx->P32.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->h_iter, ctx->P32.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ctx->pcg_last_iters += ctx->h_iter[0];
    const double bb = ctx->h_scal[4], rr = ctx->h_scal[3];
    ctx->pcg_last_rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    return MABD_OK;
  }
  run(ctx, "p32_setup", [&] { launch_p32_setup(ctx->B, ctx->J, P, rhs, rtol, ctx->d_status, s, lg, la); });
  int done = 0;
  for (int launched = 0; launched < max_it && !done; launched += PCG_CHUNK) {
    for (int i = 0; i < PCG_CHUNK; ++i)
      run(ctx, "p32_iteration", [&] { launch_p32_iteration(ctx->B, ctx->J, ctx->I, P, max_it, s, lg, la); });
    CK(cudaMemcpyAsync(ctx->h_iter, ctx->P32.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    done = ctx->h_iter[1];
  }
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->P32.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_iter, ctx->P32.iter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->pcg_last_iters += ctx->h_iter[0];
  const double bb = ctx->h_scal[4], rr = ctx->h_scal[3];
  ctx->pcg_last_rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
  run(ctx, "p32_finish", [&] { launch_p32_finish(ctx->J, P, out, learned ? nullptr : acc, s); });
  return MABD_OK;
}

// mixed-precision step on a graph: as the chain's (k_mixed.cu) with each dual
// solve an FP32 PCG solve
static mabd_status step_mixed_pcg(mabd_ctx *ctx, unsigned long long *maxbits, cudaStream_t s) {
  const StepParams &p = ctx->sp;
  ctx->pcg_last_iters = 0;
  run(ctx, "mx_body_prep", [&] {
    launch_mx_body_prep(ctx->B, p, ctx->d_status, s, maxbits ? maxbits + 3 : nullptr);
  });
  run(ctx, "mx_joint_prep", [&] { launch_mx_joint_prep(ctx->B, ctx->J, p, ctx->d_status, s); });
  if (ctx->lpc_on) {
    run(ctx, "lpc_blocks", [&] { launch_lpc_blocks(ctx->B, ctx->J, ctx->lg, ctx->la, ctx->d_status, s); });
    run(ctx, "lpc_forward", [&] { launch_lpc_forward(ctx->lg, ctx->ln, ctx->la, false, s); });
  }
  mabd_status st = p32_solve_any(ctx, s, ctx->J.b, ctx->J.lambda, nullptr);
  if (st) return st;
  const int sweeps = ctx->cfg.refine_steps;
  for (int it = 0; it < sweeps; ++it) {
    run(ctx, "mx_res_body", [&] {
      launch_mx_res_body(ctx->B, ctx->J, ctx->I, p, it == 0 ? MX_FROM_U : MX_FROM_CORRECTION, s);
    });
    unsigned long long *mb = (maxbits && it == sweeps - 1) ? maxbits + 2 : nullptr;
    run(ctx, "mx_res_joint", [&] { launch_mx_res_joint(ctx->B, ctx->J, p, mb, s); });
    st = p32_solve_any(ctx, s, ctx->J.b, ctx->J.dlam, ctx->J.lambda);
    if (st) return st;
  }
  run(ctx, "mx_final", [&] {
    launch_mx_final(ctx->B, ctx->J, ctx->I, p, sweeps == 0 ? MX_FROM_U : MX_FROM_CORRECTION, s);
  });
  if (maxbits)
    run(ctx, "residuals", [&] { launch_residuals(ctx->B, ctx->J, p, maxbits, ctx->d_status, s); });
  return MABD_OK;
}

// per-step statistics slots: max |G dq + C|, max |C(q_{n+1})|, the refinement
// residual (bit patterns of non-negative doubles), polar iterations (count)
constexpr int STAT_SLOTS = 4;

static mabd_status step_once(mabd_ctx *ctx, unsigned long long *maxbits) {
  cudaStream_t s = ctx->stream;
  if (ctx->cfg.precision != MABD_FP64 && ctx->solver == MABD_SOLVER_PCG && ctx->J.K > 0) {
    mabd_status st = step_mixed_pcg(ctx, maxbits, s);
    if (st) return st;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ctx->debug_err != cudaSuccess) e = ctx->debug_err;
    return cuda_fail(ctx, e);
  }
  enqueue_pre(ctx, s, maxbits ? maxbits + 3 : nullptr);
  if (ctx->J.K > 0 && ctx->solver == MABD_SOLVER_PCG) {
    mabd_status st = pcg_loop(ctx, s, nullptr);
    if (st) return st;
  }
  enqueue_post(ctx, maxbits, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && ctx->debug_err != cudaSuccess) e = ctx->debug_err;
  return cuda_fail(ctx, e);
}

// ---- CUDA graphs: the step's launches recorded once on a private stream ----
static cudaGraphExec_t capture(mabd_ctx *ctx, void (*body)(mabd_ctx *, cudaStream_t)) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  if (cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
  body(ctx, ctx->gstream);
  if (cudaStreamEndCapture(ctx->gstream, &g) != cudaSuccess || !g) return nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  cudaGraphDestroy(g);
  return ex;
}

static void body_pre(mabd_ctx *ctx, cudaStream_t s) { enqueue_pre(ctx, s); }
static void body_chunk(mabd_ctx *ctx, cudaStream_t s) { enqueue_pcg_chunk(ctx, s); }
static void body_post(mabd_ctx *ctx, cudaStream_t s) { enqueue_post(ctx, nullptr, s); }
static void body_step(mabd_ctx *ctx, cudaStream_t s) {
  enqueue_pre(ctx, s);
  enqueue_post(ctx, nullptr, s);
}

// builds the graphs once; on any failure graphs stay off for this context
static bool graphs_ready(mabd_ctx *ctx) {
  if (ctx->graphs_off) return false;
  if (ctx->cfg.precision != MABD_FP64 && ctx->solver == MABD_SOLVER_PCG && ctx->J.K > 0) {
    ctx->graphs_off = true;  // host-checked inner solves: launched directly
    return false;
  }
  if (ctx->graphs_built) return true;
  bool ok = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) == cudaSuccess;
  if (ok) {
    if (ctx->J.K > 0 && ctx->solver == MABD_SOLVER_PCG) {
      ctx->g_pre = capture(ctx, body_pre);
      ctx->g_chunk = capture(ctx, body_chunk);
      ctx->g_post = capture(ctx, body_post);
      ok = ctx->g_pre && ctx->g_chunk && ctx->g_post;
    } else {
      ctx->g_step = capture(ctx, body_step);
      ok = ctx->g_step != nullptr;
    }
  }
  cudaGetLastError();
  if (!ok) ctx->graphs_off = true;
  ctx->graphs_built = ok;
  return ok;
}

static mabd_status step_graph(mabd_ctx *ctx) {
  cudaStream_t gs = ctx->gstream;
  if (ctx->g_step) {
    CK(cudaGraphLaunch(ctx->g_step, gs));
    return MABD_OK;
  }
  CK(cudaGraphLaunch(ctx->g_pre, gs));
  mabd_status st = pcg_loop(ctx, gs, ctx->g_chunk);
  if (st) return st;
  CK(cudaGraphLaunch(ctx->g_post, gs));
  return MABD_OK;
}

mabd_status mabd_step(mabd_ctx *ctx, int32_t nsteps, mabd_step_stats *stats) {
  dbg_pending("enter mabd_step");
  NvtxRange range("mabd_step");
  if (!ctx || nsteps < 0) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  if (nsteps == 0) return MABD_OK;
  if (stats) {
    if (ctx->max_cap < nsteps) {
      bool ok = true;
      ctx->d_max = dnew<unsigned long long>(ctx, STAT_SLOTS * (size_t)nsteps, ok);
      if (!ok) return MABD_ERR_OUT_OF_MEMORY;
      ctx->max_cap = nsteps;
    }
    CK(cudaMemsetAsync(ctx->d_max, 0, STAT_SLOTS * (size_t)nsteps * 8, ctx->stream));
  }
  if (!stats && ctx->prof_on && !ctx->debug_sync && graphs_ready(ctx) && ctx->g_step && !ctx->g_prof &&
      ctx->prof_recs.empty()) {
    // per-launch times from replays of the step's graph with timing events
    // (captured once; a failed capture leaves the direct launches below)
    ctx->prof_capture = true;
    ctx->prof_stream = ctx->gstream;
    ctx->g_prof = capture(ctx, body_step);
    ctx->prof_capture = false;
    if (!ctx->g_prof) {
      for (auto &r : ctx->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
      ctx->prof_recs.clear();
      ctx->prof_recs.push_back(Rec{"", nullptr, nullptr});  // marks the failed attempt
    }
  }
  if (!stats && ctx->prof_on && !ctx->debug_sync && ctx->g_prof) {
    CK(cudaEventRecord(ctx->ev_in, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    for (int i = 0; i < nsteps; ++i) {
      CK(cudaGraphLaunch(ctx->g_prof, ctx->gstream));
      CK(cudaStreamSynchronize(ctx->gstream));
      for (auto &r : ctx->prof_recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        auto &acc = ctx->prof_acc[r.name];
        acc.first += ms;
        acc.second += 1;
      }
    }
    CK(cudaEventRecord(ctx->ev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
    return MABD_OK;
  }
  if (!stats && !ctx->prof_on && !ctx->debug_sync && graphs_ready(ctx)) {
    // order the private graph stream after the caller's stream and back
    CK(cudaEventRecord(ctx->ev_in, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    for (int i = 0; i < nsteps; ++i) {
      mabd_status st = step_graph(ctx);
      if (st) return st;
    }
    CK(cudaEventRecord(ctx->ev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
    return MABD_OK;
  }
  std::vector<int> pit(nsteps, 0);
  std::vector<double> prel(nsteps, 0.0);
  for (int i = 0; i < nsteps; ++i) {
    mabd_status st = step_once(ctx, stats ? ctx->d_max + STAT_SLOTS * i : nullptr);
    if (st) return st;
    if (ctx->solver == MABD_SOLVER_PCG) {
      pit[i] = ctx->pcg_last_iters;
      prel[i] = ctx->pcg_last_rel;
    }
  }
  if (!stats) return MABD_OK;
  std::vector<unsigned long long> hb(STAT_SLOTS * (size_t)nsteps);
  CK(cudaMemcpyAsync(hb.data(), ctx->d_max, hb.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < nsteps; ++i) {
    double lin, nl;
    double ref;
    std::memcpy(&lin, &hb[STAT_SLOTS * i], 8);
    std::memcpy(&nl, &hb[STAT_SLOTS * i + 1], 8);
    std::memcpy(&ref, &hb[STAT_SLOTS * i + 2], 8);
    stats[i].lin_residual = lin;
    stats[i].joint_residual = nl;
    stats[i].pcg_iters = pit[i];
    stats[i].pcg_rel_residual = prel[i];
    stats[i].refine_residual = ctx->cfg.precision != MABD_FP64 ? ref : 0.0;
    stats[i].polar_iterations = ctx->B.M > 0 ? (double)hb[STAT_SLOTS * i + 3] / ctx->B.M : 0.0;
  }
  return read_status(ctx);
}

}  // extern "C"

// device buffers of the state transfer (allocated on first use)
static mabd_status ensure_dstage(mabd_ctx *ctx) {
  if (ctx->d_stage) return MABD_OK;
  const int M = ctx->B.M;
  bool ok = true;
  double *st = dnew<double>(ctx, 24 * (size_t)std::max(M, 1), ok);
  int32_t *boi = dnew<int32_t>(ctx, std::max(M, 1), ok);
  int *flag = dnew<int>(ctx, 1, ok);
  if (!ok) return MABD_ERR_OUT_OF_MEMORY;
  if (M > 0)
    CK(cudaMemcpyAsync(boi, ctx->body_of_internal.data(), (size_t)M * 4, cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->any_frame && M > 0) {
    double *fr = dnew<double>(ctx, 9 * (size_t)M, ok);
    uint8_t *hf = dnew<uint8_t>(ctx, (size_t)M, ok);
    if (!ok) return MABD_ERR_OUT_OF_MEMORY;
    CK(cudaMemcpyAsync(fr, ctx->frames.data(), 9 * (size_t)M * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(hf, ctx->has_frame.data(), (size_t)M, cudaMemcpyHostToDevice, ctx->stream));
    ctx->d_frames = fr;
    ctx->d_has_frame = hf;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->d_stage = st;
  ctx->d_boi = boi;
  ctx->d_flag = flag;
  return MABD_OK;
}

extern "C" {

// The caller's arrays are copied to the device as given (at DMA speed when
// they are pinned) and reordered there; both calls return after the copy
// has completed, so the caller keeps ownership of its arrays.
mabd_status mabd_get_state(mabd_ctx *ctx, double *q, double *qdot) {
  dbg_pending("enter mabd_get_state");
  if (!ctx || (!q && !qdot)) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  const int M = ctx->B.M;
  mabd_status st = ensure_dstage(ctx);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  launch_state_out(ctx->B, ctx->d_boi, ctx->d_stage, s);
  if (ctx->d_frames) launch_stage_frames(ctx->d_stage, M, ctx->d_frames, ctx->d_has_frame, false, s);
  if (q) CK(cudaMemcpyAsync(q, ctx->d_stage, 12 * (size_t)M * 8, cudaMemcpyDeviceToHost, s));
  if (qdot) CK(cudaMemcpyAsync(qdot, ctx->d_stage + 12 * (size_t)M, 12 * (size_t)M * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return read_status(ctx);
}

mabd_status mabd_set_state(mabd_ctx *ctx, const double *q, const double *qdot) {
  dbg_pending("enter mabd_set_state");
  if (!ctx || !q || !qdot) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  const int M = ctx->B.M;
  mabd_status st = ensure_dstage(ctx);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  const size_t n = 12 * (size_t)M;
  CK(cudaMemcpyAsync(ctx->d_stage, q, n * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ctx->d_stage + n, qdot, n * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
  launch_state_check(ctx->d_stage, 2 * n, ctx->d_flag, s);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bad) return MABD_ERR_INVALID_ARG;  // nothing of the device state changed
  if (ctx->d_frames) launch_stage_frames(ctx->d_stage, M, ctx->d_frames, ctx->d_has_frame, true, s);
  launch_state_in(ctx->d_stage, ctx->d_boi, ctx->B, s);
  CK(cudaGetLastError());
  return MABD_OK;
}

mabd_status mabd_get_lambda(mabd_ctx *ctx, double *lambda) {
  dbg_pending("enter mabd_get_lambda");
  if (!ctx || !lambda) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  const int K = ctx->J.K;
  if (K == 0) return read_status(ctx);
  std::vector<double> hl(5 * (size_t)K);
  CK(cudaMemcpyAsync(hl.data(), ctx->J.lambda, hl.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < K; ++i) {
    const int u = ctx->joint_of_internal[i];
    const int C = joint_rows(ctx->joints[u].type);
    for (int r = 0; r < C; ++r) lambda[ctx->user_row_off[u] + r] = hl[(size_t)r * K + i];
  }
  return read_status(ctx);
}

mabd_status mabd_synchronize(mabd_ctx *ctx) {
  dbg_pending("enter mabd_synchronize");
  if (!ctx) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!ctx->frozen) {
    CK(cudaStreamSynchronize(ctx->stream));
    return MABD_OK;
  }
  return read_status(ctx);
}

mabd_status mabd_get_info(mabd_ctx *ctx, mabd_info *info) {
  if (!ctx || !info) return MABD_ERR_INVALID_ARG;
  info->bodies = (int64_t)ctx->bodies.size();
  info->joints = (int64_t)ctx->joints.size();
  int64_t rows = 0;
  for (auto &j : ctx->joints) rows += joint_rows(j.type);
  info->dual_rows = rows;
  info->topology = ctx->topology;
  info->solver = ctx->solver;
  info->device_bytes = ctx->device_bytes;
  info->precision = ctx->cfg.precision;
  info->rotation_mode = ctx->cfg.rotation_mode;
  info->jacobian_mode = ctx->cfg.jacobian_mode;
  info->refine_steps = ctx->cfg.refine_steps;
  const bool cr = ctx->solver == MABD_SOLVER_CHAIN || ctx->solver == MABD_SOLVER_LOOP;
  info->cr_levels = cr ? (int32_t)ctx->levels.size() : 0;
  info->cr_tail_level = cr ? ctx->cr_tail_level : 0;
  info->seg_levels = ctx->seg_on ? (int32_t)ctx->seg_lv.size() : 0;
  info->seg_tile = SEG_T;
  return MABD_OK;
}

mabd_status mabd_profile_enable(mabd_ctx *ctx, int32_t enable) {
  if (!ctx) return MABD_ERR_INVALID_ARG;
  ctx->prof_on = enable != 0;
  return MABD_OK;
}

mabd_status mabd_profile_reset(mabd_ctx *ctx) {
  if (!ctx) return MABD_ERR_INVALID_ARG;
  mabd_status st = harvest_profile(ctx);
  ctx->prof_acc.clear();
  return st;
}

mabd_status mabd_kernel_times(mabd_ctx *ctx, int32_t cap, const char **names, double *ms,
                              int64_t *launches, int32_t *count) {
  if (!ctx || cap < 0 || !count) return MABD_ERR_INVALID_ARG;
  mabd_status st = harvest_profile(ctx);
  if (st) return st;
  static const char *known[] = {"body_prep", "joint_prep", "chain_gram", "mx_body_prep", "mx_joint_prep",
                                "mx_chain_gram", "mx_res_body", "mx_res_joint", "cr_rhs", "mx_final",
                                "p32_setup", "p32_iteration", "p32_solve", "p32_finish", "lpc_blocks", "lpc_forward",
                                "tree_forest",
                                "cr_level", "cr_reduce", "cr_combine", "cr_tail", "loop_schur",
                                "cr_top", "cr_back", "tree_up", "tree_down", "pcg_setup",
                                "pcg_iteration", "backprop", "residuals", "seg_body", "seg_first", "seg_corr",
                                "seg_final", "seg_up"};
  int n = 0;
  for (const char *k : known) {
    auto it = ctx->prof_acc.find(k);
    if (it == ctx->prof_acc.end()) continue;
    if (n < cap) {
      if (names) names[n] = k;
      if (ms) ms[n] = it->second.first;
      if (launches) launches[n] = it->second.second;
    }
    ++n;
  }
  *count = n;
  return MABD_OK;
}

const char *mabd_error_detail(mabd_ctx *ctx) {
  if (!ctx) return "";
  return ctx->err_detail;
}

// --------------------------------------------------------------------------
// learned preconditioner
// --------------------------------------------------------------------------
}  // extern "C"

namespace {

// joint graph of a mixed-precision PCG context (ball joints only): joints
// sharing a free body are adjacent; entries sorted by (neighbour, body)
mabd_status build_lpc_graph(mabd_ctx *ctx) {
  if (ctx->lpc_graph) return MABD_OK;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  if (ctx->cfg.precision == MABD_FP64 || ctx->solver != MABD_SOLVER_PCG || ctx->J.K <= 0) {
    std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                  "the learned preconditioner needs the mixed-precision PCG path");
    return MABD_ERR_UNSUPPORTED;
  }
  const int K = ctx->J.K, M = ctx->B.M;
  struct Inc { int k, side; };
  std::vector<std::vector<Inc>> inc(M);
  std::vector<uint8_t> ones(K, 0);
  for (int k = 0; k < K; ++k) {
    const auto &d = ctx->joints[ctx->joint_of_internal[k]];
    if (d.type != MABD_JOINT_BALL) {
      std::snprintf(ctx->err_detail, sizeof(ctx->err_detail),
                    "the learned preconditioner supports ball joints only");
      return MABD_ERR_UNSUPPORTED;
    }
    int nfree = 0;
    if (!ctx->bodies[d.body_a].fixed) {
      inc[ctx->internal_of_body[d.body_a]].push_back({k, 0});
      ++nfree;
    }
    if (d.body_b >= 0 && !ctx->bodies[d.body_b].fixed) {
      inc[ctx->internal_of_body[d.body_b]].push_back({k, 1});
      ++nfree;
    }
    ones[k] = nfree == 1 ? 1 : 0;
  }
  struct Ent { int n, body; int8_t sk, sn; };
  std::vector<std::vector<Ent>> ent(K);
  for (int j = 0; j < M; ++j)
    for (const Inc &a : inc[j])
      for (const Inc &b : inc[j])
        if (a.k != b.k) ent[a.k].push_back({b.k, j, (int8_t)a.side, (int8_t)b.side});
  std::vector<int32_t> off(K + 1, 0), nbr, body, rev;
  std::vector<int8_t> sk, sn;
  for (int k = 0; k < K; ++k) {
    auto &v = ent[k];
    std::sort(v.begin(), v.end(), [](const Ent &x, const Ent &y) {
      return x.n != y.n ? x.n < y.n : x.body < y.body;
    });
    off[k + 1] = off[k] + (int)v.size();
    for (const Ent &e : v) {
      nbr.push_back(e.n);
      body.push_back(e.body);
      sk.push_back(e.sk);
      sn.push_back(e.sn);
    }
  }
  const int nnz = off[K];
  rev.assign(nnz, -1);
  for (int k = 0; k < K; ++k)
    for (int e = off[k]; e < off[k + 1]; ++e) {
      const int n = nbr[e];
      for (int f = off[n]; f < off[n + 1]; ++f)
        if (nbr[f] == k && body[f] == body[e]) {
          rev[e] = f;
          break;
        }
    }
  bool ok = true;
  const size_t nz = std::max(nnz, 1);
  int32_t *doff = dnew<int32_t>(ctx, K + 1, ok), *dnbr = dnew<int32_t>(ctx, nz, ok);
  int32_t *dbody = dnew<int32_t>(ctx, nz, ok), *drev = dnew<int32_t>(ctx, nz, ok);
  int8_t *dsk = dnew<int8_t>(ctx, nz, ok), *dsn = dnew<int8_t>(ctx, nz, ok);
  uint8_t *dones = dnew<uint8_t>(ctx, K, ok);
  LpcAct &A = ctx->la;
  A.E = dnew<float>(ctx, LPC_ES * nz, ok);
  A.C = dnew<float>(ctx, 6 * (size_t)K, ok);
  A.x = dnew<float>(ctx, LPC_F * (size_t)K, ok);
  A.h1 = dnew<float>(ctx, LPC_H * (size_t)K, ok);
  A.h2 = dnew<float>(ctx, LPC_H * (size_t)K, ok);
  A.h3 = dnew<float>(ctx, LPC_H * (size_t)K, ok);
  A.a = dnew<float>(ctx, LPC_R * (size_t)K, ok);
  A.b = dnew<float>(ctx, LPC_R * (size_t)K, ok);
  A.s = dnew<float>(ctx, K, ok);
  A.alpha = dnew<float>(ctx, nz, ok);
  ctx->P32.t = dnew<float>(ctx, 5 * (size_t)K, ok);
  ctx->P32.y = dnew<float>(ctx, 5 * (size_t)K, ok);
  DevPCGN &V = ctx->pn;
  V.r[0] = dnew<float4>(ctx, K, ok);
  V.r[1] = dnew<float4>(ctx, K, ok);
  V.p[0] = dnew<float4>(ctx, K, ok);
  V.p[1] = dnew<float4>(ctx, K, ok);
  V.q = dnew<float4>(ctx, K, ok);
  V.x = dnew<float4>(ctx, K, ok);
  V.y = dnew<float4>(ctx, K, ok);
  V.z = dnew<float4>(ctx, K, ok);
  V.cu = dnew<float>(ctx, nz, ok);
  float *dP = dnew<float>(ctx, LPC_NPARAM, ok);
  uint16_t *w1 = dnew<uint16_t>(ctx, 2 * LPC_F * LPC_H, ok), *w2 = dnew<uint16_t>(ctx, 2 * LPC_H * LPC_H, ok),
           *w3 = dnew<uint16_t>(ctx, 2 * LPC_H * LPC_H, ok);
  if (!ok) return MABD_ERR_OUT_OF_MEMORY;
  auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
  };
  CK(up(doff, off.data(), off.size() * 4));
  CK(up(dnbr, nbr.data(), nbr.size() * 4));
  CK(up(dbody, body.data(), body.size() * 4));
  CK(up(drev, rev.data(), rev.size() * 4));
  CK(up(dsk, sk.data(), sk.size()));
  CK(up(dsn, sn.data(), sn.size()));
  CK(up(dones, ones.data(), ones.size()));
  CK(cudaStreamSynchronize(ctx->stream));
  LpcGraph &G = ctx->lg;
  G.K = K;
  G.nnz = nnz;
  G.off = doff;
  G.nbr = dnbr;
  G.body = dbody;
  G.sk = dsk;
  G.sn = dsn;
  G.rev = drev;
  G.onesided = dones;
  ctx->P32.Cl = A.C;
  ctx->ln.P = dP;
  ctx->ln.W1t = w1;
  ctx->ln.W2t = w2;
  ctx->ln.W3t = w3;
  // the normalized-space solve unless MABD_PCG_NORMALIZED=0 or the device
  // cannot run a cooperative launch
  {
    const char *pe = std::getenv("MABD_PCG_NORMALIZED");
    int coop = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (coop && !(pe && pe[0] == '0')) {
      ctx->pn_nb[0] = pcgn_blocks(false);
      ctx->pn_nb[1] = pcgn_blocks(true);
    }
  }
  ctx->lpc_graph = true;
  return MABD_OK;
}

}  // namespace

// trainer: captured batches of normalized dual systems of one joint graph
struct mabd_lpc {
  cudaStream_t stream = nullptr;
  std::vector<void *> allocs;
  bool have_graph = false;
  LpcGraph g{};
  std::vector<float *> batches;  // [nnz][9] each
  LpcAct act{};
  LpcNet net{};
  float *P = nullptr, *m = nullptr, *v = nullptr;
  LpcTrainWork W{};
  float *V = nullptr;
  double *losses = nullptr;
  int losses_cap = 0;
  int nv_cap = 0;
};

namespace {

template <typename T>
T *tnew(mabd_lpc *t, size_t n, bool &ok) {
  void *p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
    return nullptr;
  }
  t->allocs.push_back(p);
  return (T *)p;
}

mabd_status lpc_alloc_work(mabd_lpc *t, int nv) {
  if (nv <= t->nv_cap) return MABD_OK;
  const size_t K = t->g.K, n3 = (size_t)nv * K * 3;
  bool ok = true;
  LpcTrainWork &W = t->W;
  t->V = tnew<float>(t, n3, ok);
  W.t = tnew<float>(t, n3, ok);
  W.u = tnew<float>(t, n3, ok);
  W.w = tnew<float>(t, n3, ok);
  W.q = tnew<float>(t, n3, ok);
  W.gw = tnew<float>(t, n3, ok);
  W.gu = tnew<float>(t, n3, ok);
  if (!ok) return MABD_ERR_OUT_OF_MEMORY;
  t->nv_cap = nv;
  return MABD_OK;
}

}  // namespace

namespace {

// forward with kept activations and the loss (and gradient) of one batch
mabd_status lpc_eval(mabd_lpc *t, int batch, int nv, const float *V, uint64_t seed, int kind, bool grad,
                     double *dloss) {
  cudaStream_t s = t->stream;
  mabd_status st = lpc_alloc_work(t, nv);
  if (st) return st;
  LpcAct A = t->act;
  A.E = t->batches[batch];
  launch_lpc_weights(t->P, (uint16_t *)t->net.W1t, (uint16_t *)t->net.W2t, (uint16_t *)t->net.W3t, s);
  launch_lpc_forward(t->g, t->net, A, true, s);
  const size_t n3 = (size_t)nv * t->g.K * 3;
  if (V) {
    if (cudaMemcpyAsync(t->V, V, n3 * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return MABD_ERR_CUDA;
  } else {
    launch_lpc_probe(t->V, n3, seed, s);
  }
  LpcTrainWork W = t->W;
  W.nv = nv;
  W.V = t->V;
  W.loss = dloss;
  launch_lpc_loss_grad(t->g, A, t->net, W, kind, grad, s);
  return cudaGetLastError() == cudaSuccess ? MABD_OK : MABD_ERR_CUDA;
}

// loss of a kind from the two sums of the loss kernels
double lpc_loss_value(int kind, const double *sums, int nv, int K) {
  const double n = (double)nv * 3.0 * K;
  return kind == 0 ? sums[0] / n : std::log(sums[0] / n) - 2.0 / K * sums[1];
}

mabd_status lpc_losses(mabd_lpc *t, int n) {
  if (n <= t->losses_cap) return MABD_OK;
  bool ok = true;
  t->losses = tnew<double>(t, 2 * (size_t)n, ok);
  if (!ok) return MABD_ERR_OUT_OF_MEMORY;
  t->losses_cap = n;
  return MABD_OK;
}

}  // namespace

extern "C" {

mabd_status mabd_tree_schedule(mabd_ctx *ctx, int32_t *counts) {
  if (!ctx || !counts) return MABD_ERR_INVALID_ARG;
  if (!ctx->frozen) return MABD_ERR_BAD_STATE;
  const int nl = (int)ctx->tree_lvl.size() - 1;
  counts[0] = std::max(nl, 0);
  counts[1] = counts[2] = 0;
  counts[3] = ctx->tree_mode;
  return MABD_OK;
}

int32_t mabd_lpc_num_params(void) { return LPC_NPARAM; }

mabd_status mabd_set_preconditioner(mabd_ctx *ctx, const float *params) {
  dbg_pending("enter mabd_set_preconditioner");
  if (!ctx) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  if (!params) {
    ctx->lpc_on = false;
    return MABD_OK;
  }
  for (int i = 0; i < LPC_NPARAM; ++i)
    if (!std::isfinite(params[i])) return MABD_ERR_INVALID_ARG;
  mabd_status st = build_lpc_graph(ctx);
  if (st) return st;
  CK(cudaMemcpyAsync((void *)ctx->ln.P, params, sizeof(float) * LPC_NPARAM, cudaMemcpyHostToDevice, ctx->stream));
  launch_lpc_weights(ctx->ln.P, (uint16_t *)ctx->ln.W1t, (uint16_t *)ctx->ln.W2t, (uint16_t *)ctx->ln.W3t,
                     ctx->stream);
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->lpc_on = true;
  return MABD_OK;
}

mabd_status mabd_lpc_fallbacks(mabd_ctx *ctx, int32_t *count) {
  if (!ctx || !count) return MABD_ERR_INVALID_ARG;
  *count = ctx->lpc_fallbacks;
  return MABD_OK;
}

mabd_status mabd_lpc_create(mabd_lpc **out) {
  if (!out) return MABD_ERR_INVALID_ARG;
  *out = nullptr;
  mabd_lpc *t = new (std::nothrow) mabd_lpc();
  if (!t) return MABD_ERR_OUT_OF_MEMORY;
  if (cudaStreamCreateWithFlags(&t->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    return MABD_ERR_CUDA;
  }
  *out = t;
  return MABD_OK;
}

mabd_status mabd_lpc_destroy(mabd_lpc *t) {
  if (!t) return MABD_ERR_INVALID_ARG;
  cudaStreamSynchronize(t->stream);
  for (void *p : t->allocs) cudaFree(p);
  cudaStreamDestroy(t->stream);
  delete t;
  return MABD_OK;
}

mabd_status mabd_lpc_capture(mabd_lpc *t, mabd_ctx *ctx, int32_t *batch) {
  dbg_pending("enter mabd_lpc_capture");
  if (!t || !ctx) return MABD_ERR_INVALID_ARG;
  if (ctx->cuda_failed) return MABD_ERR_CUDA;
  mabd_status st = build_lpc_graph(ctx);
  if (st) return st;
  cudaStream_t s = ctx->stream;
  launch_mx_body_prep(ctx->B, ctx->sp, ctx->d_status, s);
  launch_lpc_blocks(ctx->B, ctx->J, ctx->lg, ctx->la, ctx->d_status, s);
  CK(cudaStreamSynchronize(s));
  st = read_status(ctx);
  if (st) return st;
  const LpcGraph &G = ctx->lg;
  bool ok = true;
  if (!t->have_graph) {
    const size_t K = G.K, nz = std::max(G.nnz, 1);
    LpcGraph g = G;
    int32_t *off = tnew<int32_t>(t, K + 1, ok), *nbr = tnew<int32_t>(t, nz, ok), *body = tnew<int32_t>(t, nz, ok),
            *rev = tnew<int32_t>(t, nz, ok);
    int8_t *sk = tnew<int8_t>(t, nz, ok), *sn = tnew<int8_t>(t, nz, ok);
    uint8_t *ones = tnew<uint8_t>(t, K, ok);
    LpcAct &A = t->act;
    A.x = tnew<float>(t, LPC_F * K, ok);
    A.A1 = tnew<float>(t, 2 * LPC_F * K, ok);
    A.A2 = tnew<float>(t, 2 * LPC_H * K, ok);
    A.A3 = tnew<float>(t, 2 * LPC_H * K, ok);
    A.pre1 = tnew<float>(t, LPC_H * K, ok);
    A.pre2 = tnew<float>(t, LPC_H * K, ok);
    A.pre3 = tnew<float>(t, LPC_H * K, ok);
    A.h1 = tnew<float>(t, LPC_H * K, ok);
    A.h2 = tnew<float>(t, LPC_H * K, ok);
    A.h3 = tnew<float>(t, LPC_H * K, ok);
    A.a = tnew<float>(t, LPC_R * K, ok);
    A.b = tnew<float>(t, LPC_R * K, ok);
    A.s = tnew<float>(t, K, ok);
    A.alpha = tnew<float>(t, nz, ok);
    t->P = tnew<float>(t, LPC_NPARAM, ok);
    t->m = tnew<float>(t, LPC_NPARAM, ok);
    t->v = tnew<float>(t, LPC_NPARAM, ok);
    t->net.P = t->P;
    t->net.W1t = tnew<uint16_t>(t, 2 * LPC_F * LPC_H, ok);
    t->net.W2t = tnew<uint16_t>(t, 2 * LPC_H * LPC_H, ok);
    t->net.W3t = tnew<uint16_t>(t, 2 * LPC_H * LPC_H, ok);
    LpcTrainWork &W = t->W;
    W.dalpha = tnew<float>(t, nz, ok);
    W.ds = tnew<float>(t, K, ok);
    W.dh = tnew<float>(t, LPC_H * K, ok);
    W.dh2 = tnew<float>(t, LPC_H * K, ok);
    W.dA = tnew<float>(t, 2 * LPC_H * K, ok);
    W.dpre = tnew<float>(t, LPC_H * K, ok);
    W.grad = tnew<float>(t, LPC_NPARAM, ok);
    W.part = tnew<double>(t, 2 * ((K + 127) / 128) + 2, ok);
    if (!ok) return MABD_ERR_OUT_OF_MEMORY;
    CK(cudaMemcpyAsync(off, G.off, (K + 1) * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(nbr, G.nbr, nz * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(body, G.body, nz * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(rev, G.rev, nz * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(sk, G.sk, nz, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(sn, G.sn, nz, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(ones, G.onesided, K, cudaMemcpyDeviceToDevice, s));
    g.off = off;
    g.nbr = nbr;
    g.body = body;
    g.rev = rev;
    g.sk = sk;
    g.sn = sn;
    g.onesided = ones;
    t->g = g;
    t->have_graph = true;
  } else if (t->g.K != G.K || t->g.nnz != G.nnz) {
    return MABD_ERR_INVALID_ARG;  // every batch has the first context's joint graph
  }
  float *E = tnew<float>(t, LPC_ES * (size_t)std::max(G.nnz, 1), ok);
  if (!ok) return MABD_ERR_OUT_OF_MEMORY;
  CK(cudaMemcpyAsync(E, ctx->la.E, LPC_ES * (size_t)G.nnz * 4, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  t->batches.push_back(E);
  if (batch) *batch = (int32_t)t->batches.size() - 1;
  return MABD_OK;
}

mabd_status mabd_lpc_batch_blocks(mabd_lpc *t, int32_t batch, int32_t *off, int32_t *nbr, float *E) {
  if (!t || !off || !nbr || !E || !t->have_graph || batch < 0 || batch >= (int)t->batches.size())
    return MABD_ERR_INVALID_ARG;
  const LpcGraph &g = t->g;
  if (cudaMemcpyAsync(off, g.off, 4 * ((size_t)g.K + 1), cudaMemcpyDeviceToHost, t->stream) != cudaSuccess ||
      cudaMemcpyAsync(nbr, g.nbr, 4 * (size_t)g.nnz, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess ||
      cudaMemcpy2DAsync(E, 36, t->batches[batch], 4 * LPC_ES, 36, (size_t)g.nnz, cudaMemcpyDeviceToHost,
                        t->stream) != cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return MABD_ERR_CUDA;
  return MABD_OK;
}

mabd_status mabd_lpc_loss_grad(mabd_lpc *t, int32_t batch, const float *params, int32_t kind, int32_t nv,
                               const float *V, uint64_t seed, double *loss, float *grad) {
  if (!t || !params || !loss || nv < 1 || !t->have_graph || batch < 0 || batch >= (int)t->batches.size() ||
      (kind != 0 && kind != 1))
    return MABD_ERR_INVALID_ARG;
  mabd_status st = lpc_losses(t, 1);
  if (st) return st;
  if (cudaMemcpyAsync(t->P, params, sizeof(float) * LPC_NPARAM, cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
    return MABD_ERR_CUDA;
  st = lpc_eval(t, batch, nv, V, seed, kind, grad != nullptr, t->losses);
  if (st) return st;
  double l[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(l, t->losses, 16, cudaMemcpyDeviceToHost, t->stream) != cudaSuccess) return MABD_ERR_CUDA;
  if (grad && cudaMemcpyAsync(grad, t->W.grad, sizeof(float) * LPC_NPARAM, cudaMemcpyDeviceToHost, t->stream) !=
                  cudaSuccess)
    return MABD_ERR_CUDA;
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return MABD_ERR_CUDA;
  *loss = lpc_loss_value(kind, l, nv, t->g.K);
  return MABD_OK;
}

mabd_status mabd_lpc_train(mabd_lpc *t, float *params, int32_t kind, int32_t iters, float lr, int32_t nv,
                           uint64_t seed, double *losses) {
  if (!t || !params || iters < 0 || nv < 1 || !(lr > 0.f) || !t->have_graph || t->batches.empty() ||
      (kind != 0 && kind != 1))
    return MABD_ERR_INVALID_ARG;
  cudaStream_t s = t->stream;
  mabd_status st = lpc_losses(t, std::max(iters, 1));
  if (st) return st;
  if (cudaMemcpyAsync(t->P, params, sizeof(float) * LPC_NPARAM, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(t->m, 0, sizeof(float) * LPC_NPARAM, s) != cudaSuccess ||
      cudaMemsetAsync(t->v, 0, sizeof(float) * LPC_NPARAM, s) != cudaSuccess)
    return MABD_ERR_CUDA;
  const int nb = (int)t->batches.size();
  uint64_t x = seed;
  for (int it = 0; it < iters; ++it) {
    // batch order from a SplitMix64 stream of the seed
    x += 0x9E3779B97F4A7C15ULL;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    const int b = (int)(z % (uint64_t)nb);
    st = lpc_eval(t, b, nv, nullptr, z, kind, true, t->losses + 2 * it);
    if (st) return st;
    launch_lpc_adam(t->P, t->W.grad, t->m, t->v, lr, it + 1, s);
  }
  std::vector<double> hl(2 * (size_t)std::max(iters, 1));
  if (cudaMemcpyAsync(params, t->P, sizeof(float) * LPC_NPARAM, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(hl.data(), t->losses, 16 * (size_t)iters, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MABD_ERR_CUDA;
  if (losses)
    for (int i = 0; i < iters; ++i) losses[i] = lpc_loss_value(kind, &hl[2 * (size_t)i], nv, t->g.K);
  return MABD_OK;
}

mabd_status mabd_destroy(mabd_ctx *ctx) {
  dbg_pending("enter mabd_destroy");
  if (!ctx) return MABD_ERR_INVALID_ARG;
  cudaStreamSynchronize(ctx->stream);
  for (auto &r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaGraphExec_t g : {ctx->g_step, ctx->g_pre, ctx->g_chunk, ctx->g_post, ctx->g_prof})
    if (g) cudaGraphExecDestroy(g);
  for (auto &r : ctx->prof_recs) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  if (ctx->gstream) {
    cudaStreamSynchronize(ctx->gstream);
    cudaStreamDestroy(ctx->gstream);
  }
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  free_all(ctx);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->h_iter) cudaFreeHost(ctx->h_iter);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
  delete ctx;
  return MABD_OK;
}

}  // extern "C"
