// mabd_chain_step_noalloc: one chain step for callers that cannot allocate
// device memory (for example code that runs while another framework owns
// the allocator, or inside a pre-sized memory budget).  Inputs and outputs
// are the caller's device arrays; every intermediate lives in one
// file-scope __device__ array of fixed size, shared by all calls on a
// device.  The paper has no counterpart: this is a deployment variant of
// the chain path (the same step kernels as mabd_step; Hbar^{-1} is formed on
// the device by the set-up code that mabd_prefactor runs on the host).
#include <cstdio>
#include <mutex>

#include "../../include/mabd.h"
#include "mabd_device.cuh"
#include "hbar_inv.h"

namespace mabd {
namespace {

constexpr int NA_MAX_BODIES = MABD_NOALLOC_MAX_BODIES;
constexpr int NA_MAX_JOINTS = NA_MAX_BODIES + 1;
// 12.8 MB (1,600,000 doubles); carve() below checks every call's layout against it
constexpr size_t NA_SCRATCH_DOUBLES = 1600000;

static __device__ __align__(256) double g_na_scratch[NA_SCRATCH_DOUBLES];

std::mutex g_na_mutex;
void *g_na_ptr[64] = {nullptr};

struct Layout {
  DevBodies B;
  DevJoints J;
  DevIncidence I;
  DevChain C;
  CRLevel levels[32];
  int nlevels;
  double *cL, *cR, *Bn;
  int *status;
  int *bad;  // validation flag
  int8_t *jtype_rw;
  int32_t *ja_rw, *jb_rw, *ioff_rw, *ijoint_rw;
  uint8_t *jflags_rw, *fixed_rw, *flags_rw;
  int8_t *iside_rw, *islot_rw;
  double *sig_rw, *mass_rw, *vmu_rw, *vlam_rw, *hinv_rw;
  double *pa1_rw, *pb1_rw, *pa2_rw, *pb2_rw, *ua_rw;
  size_t doubles_used;
};

// Assigns every intermediate a 256-byte aligned slice of the scratch array.
bool carve(double *base, int M, int K, Layout &L) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void * {
    size_t n = (bytes + 255) / 256 * 32;  // doubles, 256-byte granules
    void *p = base + off;
    off += n;
    return p;
  };
  const size_t m = (size_t)M, k = (size_t)K, d = sizeof(double);
  // every pointer the step does not use stays null (no processing orders,
  // no mixed-form arrays)
  L.B = DevBodies{};
  L.J = DevJoints{};
  L.I = DevIncidence{};
  L.C = DevChain{};
  L.status = (int *)take(2 * sizeof(int));
  L.bad = L.status + 1;
  L.B.M = M;
  L.B.q = (double *)take(12 * m * d);
  L.B.qd = (double *)take(12 * m * d);
  L.sig_rw = (double *)take(3 * m * d);
  L.mass_rw = (double *)take(m * d);
  L.vmu_rw = (double *)take(m * d);
  L.vlam_rw = (double *)take(m * d);
  L.hinv_rw = (double *)take(HINV_N * m * d);
  L.fixed_rw = (uint8_t *)take(m);
  L.B.R = (double *)take(9 * m * d);
  L.B.ubar = (double *)take(12 * m * d);
  L.J.K = K;
  L.jtype_rw = (int8_t *)take(k);
  L.ja_rw = (int32_t *)take(4 * k);
  L.jb_rw = (int32_t *)take(4 * k);
  L.flags_rw = (uint8_t *)take(k);
  L.pa1_rw = (double *)take(3 * k * d);
  L.pb1_rw = (double *)take(3 * k * d);
  L.pa2_rw = (double *)take(3 * k * d);
  L.pb2_rw = (double *)take(3 * k * d);
  L.ua_rw = (double *)take(3 * k * d);
  L.J.RH = (double *)take(9 * k * d);
  L.J.c = (double *)take(5 * k * d);
  L.J.b = (double *)take(5 * k * d);
  L.J.lambda = (double *)take(5 * k * d);
  L.ioff_rw = (int32_t *)take(4 * (m + 1));
  L.ijoint_rw = (int32_t *)take(4 * 2 * m);
  L.iside_rw = (int8_t *)take(2 * m);
  L.islot_rw = (int8_t *)take(2 * m);
  L.C.K = K;
  L.C.off = 0;
  L.C.Dfirst = (double *)take(15 * k * d);
  L.C.Dsecond = (double *)take(15 * k * d);
  L.C.B = (double *)take(25 * k * d);
  L.jflags_rw = (uint8_t *)take(k);
  int N = K, lvl = 0;
  while (true) {
    if (lvl >= 32) return false;
    CRLevel &v = L.levels[lvl];
    v = CRLevel{};
    v.N = N;
    if (lvl > 0) {
      v.D = (double *)take(15 * (size_t)N * d);
      v.B = (double *)take(25 * (size_t)N * d);
      v.b = (double *)take(5 * (size_t)N * d);
      v.lam = (double *)take(5 * (size_t)N * d);
    } else {
      v.lam = L.J.lambda;
    }
    if (N / 2 > 0) v.fac = (double *)take(70 * (size_t)(N / 2) * d);
    ++lvl;
    if (N == 1) break;
    N = (N + 1) / 2;
  }
  L.nlevels = lvl;
  const size_t half = k / 2 > 0 ? k / 2 : 1;
  L.cL = (double *)take(20 * half * d);
  L.cR = (double *)take(20 * half * d);
  L.Bn = (double *)take(25 * half * d);
  L.doubles_used = off;
  if (off > NA_SCRATCH_DOUBLES) return false;
  L.B.sig = L.sig_rw;
  L.B.mass = L.mass_rw;
  L.B.vmu = L.vmu_rw;
  L.B.vlam = L.vlam_rw;
  L.B.hinv = L.hinv_rw;
  L.B.fixed = L.fixed_rw;
  L.J.type = L.jtype_rw;
  L.J.ja = L.ja_rw;
  L.J.jb = L.jb_rw;
  L.J.flags = L.flags_rw;
  L.J.pa1 = L.pa1_rw;
  L.J.pb1 = L.pb1_rw;
  L.J.pa2 = L.pa2_rw;
  L.J.pb2 = L.pb2_rw;
  L.J.ua = L.ua_rw;
  L.I.off = L.ioff_rw;
  L.I.joint = L.ijoint_rw;
  L.I.side = L.iside_rw;
  L.C.jflags = L.jflags_rw;
  L.C.islot = L.islot_rw;
  return true;
}

// number of incidence entries of bodies 0..j-1 of a chain with K joints
// whose first joint is a pin on body 0 iff lp = 1
__device__ __forceinline__ int na_prefix(int j, int lp, int K) {
  const int lower = lp ? j : (j > 1 ? j - 1 : 0);  // i in [0, j) with i - 1 + lp >= 0
  const int lim = K - lp > 0 ? K - lp : 0;         // i in [0, j) with i + lp < K
  const int upper = j < lim ? j : lim;
  return lower + upper;
}

// one thread per body: SoA state and constants, the chain incidence (body j
// carries the joints at positions j - 1 + lp and j + lp, lp = 1 with a pin
// on body 0) and the validation of its description
__global__ void k_na_bodies(const mabd_body_desc *bodies, int M, int K, int lp, double h,
                            DevBodies B, double *sig, double *mass, double *vmu, double *vlam,
                            double *hinv, uint8_t *fixed, int32_t *ioff, int32_t *ijoint,
                            int8_t *iside, int8_t *islot, int *bad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const mabd_body_desc &b = bodies[j];
  for (int c = 0; c < 12; ++c) {
    B.q[(size_t)c * M + j] = b.q[c];
    B.qd[(size_t)c * M + j] = b.qdot[c];
  }
  const double s[3] = {b.second_moment[0], b.second_moment[1], b.second_moment[2]};
  for (int a = 0; a < 3; ++a) sig[(size_t)a * M + j] = s[a];
  mass[j] = b.mass;
  const double mu = b.young / (2.0 * (1.0 + b.poisson));
  const double lam = b.young * b.poisson / ((1.0 + b.poisson) * (1.0 - 2.0 * b.poisson));
  vmu[j] = b.volume * mu;
  vlam[j] = b.volume * lam;
  fixed[j] = 0;
  double hv[HINV_N];
  const double tr = s[0] + s[1] + s[2];
  // the checks of mabd_add_bodies: finite, positive mass, volume, E and
  // second moment, nu in [0, 0.5), a principal frame, a finite state
  bool fin = isfinite(b.mass) && isfinite(b.volume) && isfinite(b.young) && isfinite(b.poisson);
  for (int c = 0; c < 6; ++c) fin = fin && isfinite(b.second_moment[c]);
  for (int c = 0; c < 12; ++c) fin = fin && isfinite(b.q[c]) && isfinite(b.qdot[c]);
  bool ok = fin && b.fixed == 0 && b.mass > 0.0 && b.volume > 0.0 && b.young > 0.0 && b.poisson >= 0.0 &&
            b.poisson < 0.5 && s[0] > 0.0 && s[1] > 0.0 && s[2] > 0.0 &&
            fabs(b.second_moment[3]) <= 1e-12 * tr && fabs(b.second_moment[4]) <= 1e-12 * tr &&
            fabs(b.second_moment[5]) <= 1e-12 * tr && hbar_inverse(b.mass, s, b.volume, b.young, b.poisson, h, hv);
  if (!ok) {
    atomicOr(bad, 1);
    for (int i = 0; i < HINV_N; ++i) hv[i] = 0.0;
  }
  for (int i = 0; i < HINV_N; ++i) hinv[(size_t)i * M + j] = hv[i];
  // incidence: joints at positions j-1+lp (lower) and j+lp (upper), when in
  // range; body i carries [i-1+lp >= 0] + [i+lp < K] of them, so the CSR
  // offset of body j is a closed-form prefix sum
  const int k0 = j - 1 + lp, k1 = j + lp;
  const bool has0 = k0 >= 0, has1 = k1 < K;
  const int before = na_prefix(j, lp, K);
  ioff[j] = before;
  if (j == M - 1) ioff[M] = na_prefix(M, lp, K);
  int e = before;
  if (has0) {
    ijoint[e] = k0;
    iside[e] = -1;  // resolved by k_na_joints
    islot[e] = 1;   // body j is the upper body of the joint below it
    ++e;
  }
  if (has1) {
    ijoint[e] = k1;
    iside[e] = -1;
    islot[e] = 0;
  }
}

// one thread per joint: SoA record, joint flags, the side of each incidence
// entry and the chain block flags; checks that joint k joins the bodies its
// chain position requires
__global__ void k_na_joints(const mabd_joint_desc *joints, int M, int K, int lp, DevJoints J,
                            int8_t *jtype, int32_t *ja, int32_t *jb, uint8_t *flags, double *pa1,
                            double *pb1, double *pa2, double *pb2, double *ua,
                            const int32_t *ioff, int8_t *iside, uint8_t *jflags, int *bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const mabd_joint_desc &d = joints[k];
  // chain position k joins bodies k-lp and k-lp+1; the ends may be pins
  const int lo = k - lp, hi = k - lp + 1;
  const int a = (int)d.body_a, b = (int)d.body_b;
  bool ok = d.type == 0 || d.type == 1;
  // finite points and axes (and a hinge's axis length), as mabd_add_joints requires
  for (int c = 0; c < 3; ++c)
    ok = ok && isfinite(d.anchor_a[c]) && isfinite(d.anchor_b[c]) && isfinite(d.axis_a[c]) && isfinite(d.axis_b[c]);
  if (lo < 0) ok = ok && a == 0 && b == MABD_WORLD;           // left pin on body 0
  else if (hi >= M) ok = ok && a == M - 1 && b == MABD_WORLD;  // right pin on the last body
  else ok = ok && ((a == lo && b == hi) || (a == hi && b == lo));
  double na = sqrt(d.axis_a[0] * d.axis_a[0] + d.axis_a[1] * d.axis_a[1] + d.axis_a[2] * d.axis_a[2]);
  double nb = sqrt(d.axis_b[0] * d.axis_b[0] + d.axis_b[1] * d.axis_b[1] + d.axis_b[2] * d.axis_b[2]);
  if (d.type == 1) ok = ok && na > 0.0 && nb > 0.0 && d.axis_len > 0.0 && isfinite(d.axis_len) && isfinite(na) && isfinite(nb);
  if (!ok) {
    atomicOr(bad, 1);
    return;
  }
  jtype[k] = (int8_t)d.type;
  ja[k] = a;
  jb[k] = b;
  flags[k] = (uint8_t)(JF_A_FREE | (b >= 0 ? (JF_B_BODY | JF_B_FREE) : 0));
  if (!(na > 0.0)) na = 1.0;
  if (!(nb > 0.0)) nb = 1.0;
  for (int c = 0; c < 3; ++c) {
    const double uaa = d.axis_a[c] / na, ubb = d.axis_b[c] / nb;
    pa1[(size_t)c * K + k] = d.anchor_a[c];
    pb1[(size_t)c * K + k] = d.anchor_b[c];
    ua[(size_t)c * K + k] = uaa;
    pa2[(size_t)c * K + k] = d.anchor_a[c] + d.axis_len * uaa;
    pb2[(size_t)c * K + k] = d.anchor_b[c] + d.axis_len * ubb;
  }
  // incidence sides: the entry of body x for joint k
  uint8_t jf = 0;
  for (int w = 0; w < 2; ++w) {
    const int x = w == 0 ? lo : hi;
    if (x < 0 || x >= M) continue;
    const int e = ioff[x] + (w == 0 ? ((x - 1 + lp >= 0) ? 1 : 0) : 0);
    iside[e] = (int8_t)(a == x ? 0 : 1);
    jf |= w == 0 ? 1 : 2;  // lower body writes Dfirst, upper body Dsecond
  }
  // coupling B[k] (joints k and k+1) exists when they share body hi
  if (k + 1 < K && hi < M) jf |= 4;
  jflags[k] = jf;
}

// outputs: q, qdot (12 per body, body-major) and lambda (rows, joint order)
__global__ void k_na_out(DevBodies B, DevJoints J, double *q_out, double *qd_out, double *lam_out,
                         const int32_t *row_off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B.M)
    for (int c = 0; c < 12; ++c) {
      q_out[12 * (size_t)i + c] = B.q[(size_t)c * B.M + i];
      qd_out[12 * (size_t)i + c] = B.qd[(size_t)c * B.M + i];
    }
  if (i < J.K && lam_out) {
    const int C = J.type[i] == 0 ? 3 : 5;
    const int o = row_off[i];
    for (int r = 0; r < C; ++r) lam_out[o + r] = J.lambda[(size_t)r * J.K + i];
  }
}

// lambda row offsets (exclusive prefix of 3/5) in a single thread: K <= 4097
__global__ void k_na_rowoff(DevJoints J, int32_t *row_off) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int o = 0;
  for (int k = 0; k < J.K; ++k) {
    row_off[k] = o;
    o += J.type[k] == 0 ? 3 : 5;
  }
}

}  // namespace
}  // namespace mabd

using namespace mabd;

extern "C" mabd_status mabd_chain_step_noalloc(const mabd_config *cfg, int32_t M,
                                               const mabd_body_desc *bodies, int32_t K,
                                               const mabd_joint_desc *joints, double *q_out,
                                               double *qdot_out, double *lambda_out) {
  if (!cfg || !bodies || !q_out || !qdot_out || (K > 0 && (!joints || !lambda_out)))
    return MABD_ERR_INVALID_ARG;
  if (M < 1 || M > NA_MAX_BODIES || K < 0 || K > NA_MAX_JOINTS || K < M - 1 || K > M + 1)
    return MABD_ERR_INVALID_ARG;
  if (!(cfg->h > 0.0) || cfg->precision != MABD_FP64) return MABD_ERR_INVALID_ARG;
  if (cfg->rotation_mode != MABD_ROTATION_POLAR || cfg->jacobian_mode != MABD_JACOBIAN_FROZEN)
    return MABD_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)cfg->stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return MABD_ERR_CUDA;
  }
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // the host-side name of the array is a stand-in: take its device address
      if (cudaGetSymbolAddress(&g_na_ptr[dev], g_na_scratch) != cudaSuccess) {
        cudaGetLastError();
        g_na_ptr[dev] = nullptr;
        return MABD_ERR_CUDA;
      }
    }
    base = g_na_ptr[dev];
  }
  // pin layout from the first joint: a one-sided joint there is the left pin
  int lp = 0;
  if (K == M + 1) {
    lp = 1;
  } else if (K == M) {
    mabd_joint_desc j0;
    if (cudaMemcpyAsync(&j0, joints, sizeof(j0), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return MABD_ERR_CUDA;
    }
    lp = j0.body_b == MABD_WORLD ? 1 : 0;
  }
  Layout L;
  if (!carve((double *)base, M, K, L)) return MABD_ERR_INVALID_ARG;
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(L.status, 0, 2 * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(L.J.lambda, 0, 5 * (size_t)K * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return MABD_ERR_CUDA;
  }
  StepParams p{};
  p.h = cfg->h;
  p.inv_h = 1.0 / cfg->h;
  for (int a = 0; a < 3; ++a) p.g[a] = cfg->gravity[a];
  p.residual_rhs = cfg->residual_rhs ? 1 : 0;
  const int tb = 128;
  k_na_bodies<<<(M + tb - 1) / tb, tb, 0, s>>>(bodies, M, K, lp, cfg->h, L.B, L.sig_rw, L.mass_rw,
                                               L.vmu_rw, L.vlam_rw, L.hinv_rw, L.fixed_rw, L.ioff_rw,
                                               L.ijoint_rw, L.iside_rw, L.islot_rw, L.bad);
  if (K > 0)
    k_na_joints<<<(K + tb - 1) / tb, tb, 0, s>>>(joints, M, K, lp, L.J, L.jtype_rw, L.ja_rw, L.jb_rw,
                                                 L.flags_rw, L.pa1_rw, L.pb1_rw, L.pa2_rw, L.pb2_rw,
                                                 L.ua_rw, L.ioff_rw, L.iside_rw, L.jflags_rw, L.bad);
  int flags[2] = {0, 0};
  if (cudaMemcpyAsync(flags, L.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MABD_ERR_CUDA;
  }
  if (flags[1]) return MABD_ERR_INVALID_ARG;
  // the step: the same kernels as mabd_step on a chain
  launch_body_prep(L.B, p, L.status, s);
  if (K > 0) {
    launch_joint_prep(L.B, L.J, p, L.status, s);
    launch_chain_gram(L.B, L.J, L.I, L.C, s);
    for (int l = 0; l + 1 < L.nlevels; ++l) {
      launch_cr_reduce(L.C, L.J, L.levels[l], l, L.cL, L.cR, L.Bn, L.status, s);
      launch_cr_combine(L.C, L.J, L.levels[l], l, L.levels[l + 1], L.cL, L.cR, L.Bn, s);
    }
    launch_cr_top(L.C, L.J, L.levels[L.nlevels - 1], L.nlevels - 1, L.status, s);
    for (int l = L.nlevels - 2; l >= 0; --l) launch_cr_back(L.C, L.J, L.levels[l], L.levels[l + 1], l, s);
  }
  launch_backprop(L.B, L.J, L.I, p, L.status, s);
  int32_t *row_off = (int32_t *)L.cL;  // the reduction scratch is free again
  if (K > 0) k_na_rowoff<<<1, 32, 0, s>>>(L.J, row_off);
  const int n = M > K ? M : K;
  k_na_out<<<(n + tb - 1) / tb, tb, 0, s>>>(L.B, L.J, q_out, qdot_out, K > 0 ? lambda_out : nullptr,
                                            row_off);
  if (cudaGetLastError() != cudaSuccess) return MABD_ERR_CUDA;
  if (cudaMemcpyAsync(flags, L.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MABD_ERR_CUDA;
  }
  const int bits = flags[0];
  if (bits & ST_INVERTED) return MABD_ERR_INVERTED;
  if (bits & ST_NONFINITE) return MABD_ERR_NONFINITE;
  if (bits & ST_NOT_SPD) return MABD_ERR_NOT_SPD;
  if (bits & ST_POLAR_NOCONV) return MABD_ERR_NO_CONVERGENCE;
  return MABD_OK;
}
