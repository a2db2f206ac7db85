// mlmc_api.cu -- the C ABI declared in include/mlmc.h: parameter checks,
// workspace layout, the fixed-order reductions, and the host-driven MLMC and
// plain Monte Carlo drivers.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <nvtx3/nvToolsExt.h>
#include <utility>

#include "mlmc_internal.h"
#include "mlmc_reduce.cuh"

// NVTX ranges name the host-side phases in a profiler's timeline (a no-op
// unless a tool is attached).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace mlmc {

// Launchers exported by the kernel translation units: prec_f32 / prec_f64
// hold every kernel; prec_f32_b3 / prec_f32_b4 / prec_f32_x2 / prec_f32_x2b3
// hold the level-sums and persistent kernels of the other tuning variants
// (tighter register budgets; two path pairs per thread).
#define MLMC_DECLARE_MULTI(NS)                                                                 \
  namespace NS {                                                                               \
  cudaError_t multilevel(int, const HostModel&, const ReqPlan*, int, uint32_t, Partial*,      \
                         unsigned int*, int, cudaStream_t);                                     \
  cudaError_t multilevel_dev(int, const HostModel&, const DevPlan*, Partial*, unsigned int*,  \
                             int, cudaStream_t);                                                \
  cudaError_t multilevel_table(int, const void*, size_t, const PlanReq*, int, uint32_t,       \
                               Partial*, unsigned int*, int, cudaStream_t);                     \
  int occupancy_multi(int);                                                                    \
  int occupancy_sums(int);                                                                     \
  cudaError_t level_sums(int, const HostModel&, const LevelSpec&, uint64_t, uint64_t,         \
                         Partial*, int, cudaStream_t);                                          \
  cudaError_t paths_variant(int, const HostModel&, const LevelSpec&, uint64_t, uint64_t,      \
                            void*, int32_t*, cudaStream_t);                                     \
  }
#define MLMC_DECLARE_ALL(NS)                                                                   \
  MLMC_DECLARE_MULTI(NS)                                                                       \
  namespace NS {                                                                               \
  size_t model_size();                                                                         \
  void model_image(const HostModel&, void*);                                                   \
  cudaError_t paths(int, const HostModel&, const LevelSpec&, uint64_t, uint64_t, void*,       \
                    int32_t*, void*, void*, void*, void*, bool, cudaStream_t);                  \
  int occupancy(int, bool);                                                                    \
  cudaError_t pdf(int, const HostModel&, const LevelSpec&, uint64_t, uint64_t, int, double*,  \
                  int, cudaStream_t);                                                           \
  }
MLMC_DECLARE_ALL(prec_f32)
MLMC_DECLARE_ALL(prec_f64)
MLMC_DECLARE_MULTI(prec_f32_b3)
MLMC_DECLARE_MULTI(prec_f32_b4)
MLMC_DECLARE_MULTI(prec_f32_x2)
MLMC_DECLARE_MULTI(prec_f32_x2b3)

// ---------------------------------------------------------------------------
// Tuning table of the persistent kernels per (integrator, precision):
// register-budget variant (resident blocks per SM the kernel is compiled
// for: 1 = uncapped, 3, 4; 12 and 13 = two path pairs per thread on the
// packed FP32 instructions, compiled for 2 or 3 blocks per SM; FP64 has
// only 1),
// work items per resident block
// in the planner, and resident blocks per SM actually launched (0 = as many
// as fit).  The defaults are the best of a GB300 sweep; the autotuner
// (paper_1612_07717_gb300/autotune.py) replaces them.
// ---------------------------------------------------------------------------
struct Tune {
  int variant, items_per_block, blocks_per_sm;
};
static Tune g_tune[3][2] = {{{12, 32, 0}, {1, 4, 0}},   // SE
                            {{13, 32, 0}, {1, 4, 0}},   // GL
                            {{13, 32, 0}, {1, 4, 0}}};  // BAOAB
static std::mutex g_tune_mu;

static Tune tune_of(int prec, int integ) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune[integ][prec];
}

int items_per_block(int prec, int integ) { return tune_of(prec, integ).items_per_block; }
uint64_t min_item_paths(int prec, int integ) {
  return (uint64_t)kBlock * (tune_of(prec, integ).variant >= 12 ? 2u : 1u);
}

#define MLMC_DISPATCH_VARIANT(prec, variant, CALL)                 \
  do {                                                             \
    if (prec) return prec_f64::CALL;                               \
    switch (variant) {                                             \
      case 3: return prec_f32_b3::CALL;                            \
      case 4: return prec_f32_b4::CALL;                            \
      case 12: return prec_f32_x2::CALL;                           \
      case 13: return prec_f32_x2b3::CALL;                         \
      default: return prec_f32::CALL;                              \
    }                                                              \
  } while (0)
#define MLMC_DISPATCH_MULTI(prec, integ, CALL) \
  MLMC_DISPATCH_VARIANT(prec, tune_of(prec, integ).variant, CALL)

cudaError_t launch_level_sums(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                              uint64_t N, uint64_t offset, Partial* partials, int grid,
                              cudaStream_t st) {
  if (hm.adapt) return launch_adapt_sums(prec, integ, hm, lv, N, offset, partials, grid, st);
  MLMC_DISPATCH_MULTI(prec, integ, level_sums(integ, hm, lv, N, offset, partials, grid, st));
}
cudaError_t launch_multilevel(int prec, int integ, const HostModel& hm, const ReqPlan* plan,
                              int n_req, uint32_t n_items, Partial* partials,
                              unsigned int* counter, int grid, cudaStream_t st) {
  if (hm.adapt)
    return launch_adapt_multilevel(prec, integ, hm, plan, n_req, n_items, partials, counter, grid,
                                   st);
  MLMC_DISPATCH_MULTI(prec, integ,
                      multilevel(integ, hm, plan, n_req, n_items, partials, counter, grid, st));
}
cudaError_t launch_multilevel_dev(int prec, int integ, const HostModel& hm, const DevPlan* plan,
                                  Partial* partials, unsigned int* counter, int grid,
                                  cudaStream_t st) {
  MLMC_DISPATCH_MULTI(prec, integ, multilevel_dev(integ, hm, plan, partials, counter, grid, st));
}
cudaError_t launch_multilevel_table(int prec, int integ, const void* models, size_t stride,
                                   const PlanReq* reqs, int n_req, uint32_t n_items,
                                   Partial* partials, unsigned int* counter, int grid,
                                   cudaStream_t st) {
  MLMC_DISPATCH_MULTI(prec, integ, multilevel_table(integ, models, stride, reqs, n_req, n_items,
                                                    partials, counter, grid, st));
}
static int occupancy_multi(int prec, int integ) {
  MLMC_DISPATCH_MULTI(prec, integ, occupancy_multi(integ));
}
cudaError_t launch_multilevel_table_variant(int variant, int prec, int integ, const void* models,
                                            size_t stride, const PlanReq* reqs, int n_req,
                                            uint32_t n_items, Partial* partials,
                                            unsigned int* counter, int grid, cudaStream_t st) {
  MLMC_DISPATCH_VARIANT(prec, variant, multilevel_table(integ, models, stride, reqs, n_req,
                                                        n_items, partials, counter, grid, st));
}
static int occupancy_variant(int variant, int prec, int integ) {
  MLMC_DISPATCH_VARIANT(prec, variant, occupancy_multi(integ));
}
static int occupancy_sums(int prec, int integ) {
  MLMC_DISPATCH_MULTI(prec, integ, occupancy_sums(integ));
}
size_t model_bytes(int prec) { return prec ? prec_f64::model_size() : prec_f32::model_size(); }
void model_image(int prec, const HostModel& hm, void* out) {
  if (prec) prec_f64::model_image(hm, out);
  else prec_f32::model_image(hm, out);
}
cudaError_t launch_paths(int prec, int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N,
                         uint64_t offset, void* s, int32_t* f, cudaStream_t st) {
  if (hm.adapt) return launch_adapt_paths(prec, integ, hm, lv, N, offset, s, f, nullptr, st);
  return prec ? prec_f64::paths(integ, hm, lv, N, offset, s, f, nullptr, nullptr, nullptr, nullptr,
                                false, st)
              : prec_f32::paths(integ, hm, lv, N, offset, s, f, nullptr, nullptr, nullptr, nullptr,
                                false, st);
}
// Final states through the path code of one tuning variant (variant 0: the
// table's variant for this integrator and precision).
static cudaError_t launch_paths_variant(int variant, int prec, int integ, const HostModel& hm,
                                        const LevelSpec& lv, uint64_t N, uint64_t offset, void* s,
                                        int32_t* f, cudaStream_t st) {
  if (variant == 0) variant = tune_of(prec, integ).variant;
  MLMC_DISPATCH_VARIANT(prec, variant, paths_variant(integ, hm, lv, N, offset, s, f, st));
}
cudaError_t launch_trace(int prec, int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N,
                         uint64_t offset, void* tf, void* tc, void* thf, void* thc,
                         cudaStream_t st) {
  return prec ? prec_f64::paths(integ, hm, lv, N, offset, nullptr, nullptr, tf, tc, thf, thc, true,
                                st)
              : prec_f32::paths(integ, hm, lv, N, offset, nullptr, nullptr, tf, tc, thf, thc, true,
                                st);
}
cudaError_t launch_pdf(int prec, int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N,
                       uint64_t offset, int k, double* partials, int grid, cudaStream_t st) {
  return prec ? prec_f64::pdf(integ, hm, lv, N, offset, k, partials, grid, st)
              : prec_f32::pdf(integ, hm, lv, N, offset, k, partials, grid, st);
}
int blocks_per_sm(int prec, int integ, bool multilevel) {
  if (!multilevel) return occupancy_sums(prec, integ);
  int nb = occupancy_multi(prec, integ);
  const int want = tune_of(prec, integ).blocks_per_sm;
  if (want > 0 && want < nb) nb = want;
  return nb;
}

// ---------------------------------------------------------------------------
// Fixed-order reductions of block / item partials into mlmc_level_result.
// One block per result; thread t takes partials t, t + 256, ... with Kahan
// compensation, then the same warp tree and warp-ordered Kahan sum, one lane
// of warp 0 per sum (FP64 instructions hold the FP64 pipe for many cycles
// whatever the number of active lanes, so the sums go side by side).  A warp
// none of whose threads took a partial skips its tree: its sums are zeros.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kadd(double& s, double& c, double x) {
  const double y = x - c;
  const double t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ void reduce_range(const Partial* __restrict__ p, uint32_t begin, uint32_t end,
                             uint64_t path_steps, mlmc_level_result* __restrict__ out) {
  __shared__ double s_tree[kBlock / 32][12][16];
  __shared__ unsigned long long s_u[kBlock / 32][3];
  double s[12], c[12];
  for (int k = 0; k < 12; ++k) s[k] = c[k] = 0.0;
  unsigned long long u[3] = {0, 0, 0};
  for (uint32_t j = begin + threadIdx.x; j < end; j += kBlock) {
    for (int k = 0; k < 6; ++k) kadd(s[k], c[k], p[j].s0[k]);
    for (int k = 0; k < 6; ++k) kadd(s[6 + k], c[6 + k], p[j].s1[k]);
    u[0] += p[j].n;
    u[1] += p[j].bad;
    u[2] += p[j].steps;
  }
  double v[12];
  for (int k = 0; k < 12; ++k) v[k] = s[k] - c[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (begin + (uint32_t)(warp * 32) < end) {
    warp_tree12(v, s_tree[warp], lane);
    for (int off = 16; off > 0; off >>= 1)
      for (int k = 0; k < 3; ++k) u[k] += __shfl_down_sync(0xFFFFFFFFu, u[k], off);
  } else if (lane < 12) {
    s_tree[warp][lane][0] = 0.0;
  }
  if (lane == 0)
    for (int k = 0; k < 3; ++k) s_u[warp][k] = u[k];
  __syncthreads();
  if (threadIdx.x < 12) {
    const int k = threadIdx.x;
    double t = 0.0, tc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) kadd(t, tc, s_tree[w][k][0]);
    out->sum[k / 6][k % 6] = t - tc;
  } else if (threadIdx.x < 15) {
    const int k = threadIdx.x - 12;
    unsigned long long q = 0;
    for (int w = 0; w < kBlock / 32; ++w) q += s_u[w][k];
    if (k == 0) out->n = q;
    else if (k == 1) out->n_nonfinite = q;
    else out->path_steps = path_steps ? path_steps : q;  // fixed counts come from the host
  } else if (threadIdx.x == 15) {
    out->reserved = 0;
  }
}

__global__ void __launch_bounds__(kBlock) k_finalize(const Partial* __restrict__ p, uint32_t nb,
                                                     uint64_t path_steps,
                                                     mlmc_level_result* __restrict__ out) {
  reduce_range(p, 0, nb, path_steps, out);
}

struct FinalizeMultiArgs {
  uint32_t begin[kMaxReq], end[kMaxReq];
  uint64_t path_steps[kMaxReq];
};

__global__ void __launch_bounds__(kBlock) k_finalize_multi(const Partial* __restrict__ p,
                                                           const __grid_constant__ FinalizeMultiArgs a,
                                                           mlmc_level_result* __restrict__ out) {
  const int r = blockIdx.x;
  reduce_range(p, a.begin[r], a.end[r], a.path_steps[r], out + r);
}

// Reduction of a device-planned launch: one block per planned request.
__global__ void __launch_bounds__(kBlock) k_finalize_dev(const Partial* __restrict__ p,
                                                         const DevPlan* __restrict__ plan,
                                                         mlmc_level_result* __restrict__ out) {
  const int r = blockIdx.x;
  if (r >= plan->n_req) return;
  const PlanReq& q = plan->req[r];
  reduce_range(p, q.item_base, q.item_base + q.n_items, q.path_steps, out + r);
}

cudaError_t launch_finalize_dev(const Partial* partials, const DevPlan* plan,
                                mlmc_level_result* d_out, cudaStream_t st) {
  k_finalize_dev<<<kMaxReq, kBlock, 0, st>>>(partials, plan, d_out);
  return cudaGetLastError();
}

// Reduction of a request table: one block per request.
__global__ void __launch_bounds__(kBlock) k_finalize_table(const Partial* __restrict__ p,
                                                           const PlanReq* __restrict__ reqs,
                                                           mlmc_level_result* __restrict__ out) {
  const PlanReq& q = reqs[blockIdx.x];
  reduce_range(p, q.item_base, q.item_base + q.n_items, q.path_steps, out + blockIdx.x);
}

cudaError_t launch_finalize_table(const Partial* partials, const PlanReq* reqs, int n_req,
                                  mlmc_level_result* d_out, cudaStream_t st) {
  if (n_req <= 0) return cudaSuccess;
  k_finalize_table<<<n_req, kBlock, 0, st>>>(partials, reqs, d_out);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Partial* partials, int nblocks, uint64_t path_steps,
                            mlmc_level_result* d_out, cudaStream_t st) {
  k_finalize<<<1, kBlock, 0, st>>>(partials, (uint32_t)nblocks, path_steps, d_out);
  return cudaGetLastError();
}

cudaError_t launch_finalize_multi(const Partial* partials, const ReqPlan* plan, int n_req,
                                  mlmc_level_result* d_out, cudaStream_t st) {
  FinalizeMultiArgs a;
  for (int r = 0; r < n_req; ++r) {
    a.begin[r] = plan[r].item_base;
    a.end[r] = plan[r].item_base + plan[r].n_items;
    a.path_steps[r] = plan[r].path_steps;
  }
  k_finalize_multi<<<n_req, kBlock, 0, st>>>(partials, a, d_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Parameter checks and derived constants
// ---------------------------------------------------------------------------
// lambda = 1 / tau of the regularised profile (Eq. profiles with the cut-off
// of Eq. regularisation): sigma_w(z_c) (1 / z_c + c_f f / u*) / kappa_tau.
static double lambda_at(const HostModel& hm, double z) {
  const double zc = std::fmin(std::fmax(z, hm.eps), hm.H - hm.eps);
  const double sig = hm.A * std::pow(1.0 - zc / hm.H, 0.75);
  return sig * (1.0 / zc + hm.cfu) * hm.inv_ktau;
}

int make_host_model(const mlmc_params* p, uint64_t seed, HostModel* hm) {
  if (!p) return MLMC_EINVAL;
  const double us = p->u_star;
  if (!(us > 0.0) || !(p->kappa_sigma > 0.0) || !(p->kappa_tau > 0.0)) return MLMC_EINVAL;
  if (!(p->f_coriolis >= 0.0) || !(p->c_f >= 0.0)) return MLMC_EINVAL;
  double H = p->H;
  if (!(H > 0.0)) {
    if (!(p->f_coriolis > 0.0)) return MLMC_EINVAL;
    H = 0.3 * us / p->f_coriolis;
  }
  if (!std::isfinite(H)) return MLMC_EINVAL;
  if (!(p->eps_reg_frac > 0.0) || !(p->eps_reg_frac <= 0.5)) return MLMC_EINVAL;
  if (!(p->T > 0.0) || !std::isfinite(p->T)) return MLMC_EINVAL;
  if (p->M0 < 1 || p->level_min < 0 || p->level_min > 40) return MLMC_EINVAL;
  if (p->w0_mode < 0 || p->w0_mode > 2) return MLMC_EINVAL;
  if (p->w0_mode != 2 && !(p->z0 >= 0.0 && p->z0 <= H)) return MLMC_EINVAL;
  if (!std::isfinite(p->w0) || !std::isfinite(p->qoi_threshold)) return MLMC_EINVAL;
  if (p->coupling < 0 || p->coupling > 1) return MLMC_EINVAL;
  if (p->drift_outside < 0 || p->drift_outside > 1) return MLMC_EINVAL;
  if (p->precision != MLMC_FP32 && p->precision != MLMC_FP64) return MLMC_EINVAL;
  if (p->qoi1_mode < 0 || p->qoi1_mode > 1) return MLMC_EINVAL;
  hm->qoi1_mode = p->qoi1_mode;
  hm->smooth_r = p->smooth_r;
  hm->qa = p->qoi_a;
  hm->qb = p->qoi_b;
  hm->delta = p->smooth_delta;
  for (int k = 0; k < kMaxSmoothR + 2; ++k) hm->pc[k] = 0.0;
  if (p->qoi1_mode == 1 || p->smooth_delta > 0.0) {
    if (p->smooth_r < 0 || p->smooth_r > kMaxSmoothR) return MLMC_EINVAL;
    if (!(p->smooth_delta > 0.0) || !std::isfinite(p->smooth_delta)) return MLMC_EINVAL;
    if (p->qoi1_mode == 1 &&
        (!(p->qoi_a < p->qoi_b) || !std::isfinite(p->qoi_a) || !std::isfinite(p->qoi_b)))
      return MLMC_EINVAL;
    if (smooth_coefficients(p->smooth_r, hm->pc) != 0) return MLMC_EINVAL;
  }
  const double A = p->kappa_sigma * us;
  hm->H = H;
  hm->eps = p->eps_reg_frac * H;
  hm->A = A;
  hm->inv_ktau = 1.0 / p->kappa_tau;
  hm->cfu = p->c_f * p->f_coriolis / us;
  hm->hD = -0.75 * A * A / H;
  hm->hDs = -0.75 / H;
  hm->qthr = p->qoi_threshold;
  hm->z0 = p->z0;
  hm->w0 = p->w0;
  hm->T = p->T;
  hm->w0_mode = p->w0_mode;
  hm->coupling = p->coupling;
  hm->drift_outside = p->drift_outside;
  hm->M0 = p->M0;
  hm->level_min = p->level_min;
  hm->stream_id = p->stream_id;
  // Adaptive timesteps (Section 7.2): lambda(X_adapt) of the regularised
  // profile; the bound on lambda_max / lambda(X_adapt) bounds the steps per
  // path (at most 1024 M per path).
  if (!(p->z_adapt >= 0.0) || !(p->z_adapt <= H)) return MLMC_EINVAL;
  hm->adapt = p->z_adapt > 0.0 ? 1 : 0;
  hm->z_adapt = p->z_adapt;
  hm->lam_a = 0.0;
  if (hm->adapt) {
    if (p->M0 > (1 << 22)) return MLMC_EINVAL;
    hm->lam_a = lambda_at(*hm, p->z_adapt);
    if (!(hm->lam_a * 1024.0 >= lambda_at(*hm, 0.0))) return MLMC_EINVAL;
  }
  // Philox round keys: the key schedule adds the Weyl constants per round.
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    hm->rk0[r] = k0;
    hm->rk1[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return MLMC_OK;
}

int level_spec(const HostModel& hm, int level, LevelSpec* ls) {
  if (level < hm.level_min || level > 40) return MLMC_EINVAL;
  const int64_t M = (int64_t)hm.M0 << level;
  if (M <= 0 || M > ((int64_t)1 << 40)) return MLMC_EINVAL;
  ls->level = level;
  ls->M = M;
  ls->h = hm.T / (double)M;
  ls->coupled = level > hm.level_min;
  if (ls->coupled && (M & 1)) return MLMC_EINVAL;
  return MLMC_OK;
}

// Smoothing polynomial of Section 5.1: p_r has degree r + 1, p(-1) = 1,
// p(1) = 0 and the first r moments of the step function on [-1, 1].  The
// conditions are invariant under s -> -s, p -> 1 - p, so the unique solution
// is p(s) = 1/2 - q(s) with q odd: q(s) = sum_{k odd <= r+1} b_k s^k,
//   q(1) = 1/2,   int_{-1}^{1} s^j q(s) ds = 1 / (j + 1) for odd j < r
// (even moments hold by symmetry).  Solved by Gaussian elimination.
int smooth_coefficients(int r, double* c) {
  if (r < 0 || r > kMaxSmoothR) return -1;
  int ks[kMaxSmoothR + 2], n = 0;
  for (int k = 1; k <= r + 1; k += 2) ks[n++] = k;
  double A[kMaxSmoothR][kMaxSmoothR + 1];
  int row = 0;
  for (int i = 0; i < n; ++i) A[row][i] = 1.0;           // q(1) = 1/2
  A[row][n] = 0.5;
  ++row;
  for (int j = 1; j < r && row < n; j += 2, ++row) {     // odd moments
    for (int i = 0; i < n; ++i) A[row][i] = 2.0 / (double)(j + ks[i] + 1);
    A[row][n] = 1.0 / (double)(j + 1);
  }
  if (row != n) return -1;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (std::fabs(A[i][col]) > std::fabs(A[piv][col])) piv = i;
    if (A[piv][col] == 0.0) return -1;
    for (int k = 0; k <= n; ++k) std::swap(A[col][k], A[piv][k]);
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      const double f = A[i][col] / A[col][col];
      for (int k = col; k <= n; ++k) A[i][k] -= f * A[col][k];
    }
  }
  for (int k = 0; k < kMaxSmoothR + 2; ++k) c[k] = 0.0;
  c[0] = 0.5;
  for (int i = 0; i < n; ++i) c[ks[i]] = -A[i][n] / A[i][i];
  return 0;
}

// lambda is largest at the regularisation height (it falls with z).
static double lambda_max(const HostModel& hm) { return lambda_at(hm, hm.eps); }

uint64_t steps_per_pair(const LevelSpec& ls) {
  return ls.coupled ? (uint64_t)(ls.M + ls.M / 2) : (uint64_t)ls.M;
}

// ---------------------------------------------------------------------------
// Device facts and workspace layout
//   [0, 256)                  header: work counter
//   [256, 256 + 32 * 128)     results of up to kMaxReq requests
//   [..., + P * 128)          partials, P = max(blocks of one grid, kMaxItems)
// ---------------------------------------------------------------------------
static DevInfo g_dev[64];
static std::mutex g_mu;

int device_info(DevInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MLMC_ENODEV;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev[dev].sms == 0) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return MLMC_ENODEV;
    g_dev[dev].sms = prop.multiProcessorCount;
    g_dev[dev].cc = prop.major * 10 + prop.minor;
  }
  *out = g_dev[dev];
  return MLMC_OK;
}

static constexpr size_t kHeader = 256;
static constexpr size_t kResults = (size_t)kMaxReq * sizeof(mlmc_level_result);
static constexpr size_t kMaxGridBlocks = 4096;  // >= SMs * kMaxBlocksPerSM on GB300
static size_t partial_slots() {
  return kMaxGridBlocks > (size_t)kMaxItems ? kMaxGridBlocks : (size_t)kMaxItems;
}
size_t workspace_needed() {
  return kHeader + kResults + partial_slots() * sizeof(Partial) + kGraphRegion;
}

int carve(void* ws, size_t bytes, Workspace* w) {
  if (!ws || ((uintptr_t)ws & 255) != 0 || bytes < workspace_needed()) return MLMC_EWORKSPACE;
  char* b = (char*)ws;
  w->counter = (unsigned int*)b;
  w->results = (mlmc_level_result*)(b + kHeader);
  w->partials = (Partial*)(b + kHeader + kResults);
  w->graph = b + kHeader + kResults + partial_slots() * sizeof(Partial);
  return MLMC_OK;
}

int grid_for(int prec, int integ, bool multilevel, uint64_t N) {
  DevInfo di;
  if (device_info(&di) != MLMC_OK) return 0;
  int g = di.sms * blocks_per_sm(prec, integ, multilevel);
  if ((size_t)g > kMaxGridBlocks) g = (int)kMaxGridBlocks;
  if (!multilevel) {
    const uint64_t per_block = min_item_paths(prec, integ);  // pairs of one pass of a block
    const uint64_t need = (N + per_block - 1) / per_block;
    if (need < (uint64_t)g) g = (int)(need > 0 ? need : 1);
  }
  return g;
}

int grid_for_variant(int variant, int prec, int integ) {
  DevInfo di;
  if (device_info(&di) != MLMC_OK) return 0;
  int g = di.sms * occupancy_variant(variant, prec, integ);
  if ((size_t)g > kMaxGridBlocks) g = (int)kMaxGridBlocks;
  return g;
}

// Grid of the adaptive multi-level kernel: its own occupancy (its chunk's
// shared memory and registers), whatever uniform variant is tuned.
static int grid_adapt_multi(int prec, int integ) {
  DevInfo di;
  if (device_info(&di) != MLMC_OK) return 0;
  int g = di.sms * adapt_multi_blocks_per_sm(prec, integ);
  if ((size_t)g > kMaxGridBlocks) g = (int)kMaxGridBlocks;
  return g;
}

// Grid of the adaptive level-sums kernel: blocks take contiguous pair ranges,
// as many blocks as the kernel keeps resident (its own registers and chunk).
static int grid_adapt(int prec, int integ, uint64_t N) {
  DevInfo di;
  if (device_info(&di) != MLMC_OK) return 0;
  int g = di.sms * adapt_sums_blocks_per_sm(prec, integ);
  if ((size_t)g > kMaxGridBlocks) g = (int)kMaxGridBlocks;
  const uint64_t need = (N + kBlock - 1) / kBlock;
  if (need < (uint64_t)g) g = (int)(need > 0 ? need : 1);
  return g;
}

// Adaptive timesteps exist for SE and GL only (Section 7.2); with them every
// step has h_n lambda(X_n) <= h lambda(X_adapt), so SE's bound uses
// lambda(X_adapt) in place of lambda_max.
int check_stable(int integ, const mlmc_params* p, const HostModel& hm, const LevelSpec& ls) {
  if (hm.adapt && integ == MLMC_BAOAB) return MLMC_EINVAL;
  if (hm.adapt && ls.M > kAdaptMaxM) return MLMC_EINVAL;
  if (integ != MLMC_SE || p->allow_unstable) return MLMC_OK;
  const double hmax = ls.coupled ? 2.0 * ls.h : ls.h;  // the coarse path steps 2h
  const double lam = hm.adapt ? hm.lam_a : lambda_max(hm);
  return lam * hmax < 2.0 ? MLMC_OK : MLMC_EUNSTABLE;
}

// Steps of N pairs when they are fixed (uniform timesteps); 0 asks the
// reduction for the steps the adaptive kernels counted.
static uint64_t fixed_steps(const HostModel& hm, const LevelSpec& ls, uint64_t N) {
  return hm.adapt ? 0 : N * steps_per_pair(ls);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? MLMC_OK : MLMC_ECUDA; }

// Eight independent FMA chains per thread; the operands come from memory so
// nothing folds, and the results are stored so nothing is dropped.
__global__ void __launch_bounds__(kBlock) k_ffma_probe(float* __restrict__ buf, int iters) {
  const int t = blockIdx.x * kBlock + threadIdx.x;
  const float b = buf[(t * 7) & 1023] * 1e-30f + 0.999f;
  const float c = buf[(t * 13) & 1023] * 1e-30f + 1e-3f;
  float a0 = t, a1 = t + 1, a2 = t + 2, a3 = t + 3, a4 = t + 4, a5 = t + 5, a6 = t + 6, a7 = t + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, b, c); a1 = fmaf(a1, b, c); a2 = fmaf(a2, b, c); a3 = fmaf(a3, b, c);
      a4 = fmaf(a4, b, c); a5 = fmaf(a5, b, c); a6 = fmaf(a6, b, c); a7 = fmaf(a7, b, c);
    }
  }
  buf[1024 + (t & ((1 << 20) - 1025))] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace mlmc

using namespace mlmc;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* mlmc_strerror(int code) {
  switch (code) {
    case MLMC_OK: return "success";
    case MLMC_EINVAL: return "invalid argument or parameter";
    case MLMC_EWORKSPACE: return "workspace missing, not 256-byte aligned, or too small";
    case MLMC_ECUDA: return "CUDA call failed";
    case MLMC_ENONFINITE: return "some paths diverged and were excluded";
    case MLMC_ETIMEOUT: return "device work loop hit its iteration limit";
    case MLMC_EUNSTABLE: return "symplectic Euler is unstable at this timestep (h lambda_max >= 2)";
    case MLMC_ENOTCONV: return "adaptive driver reached L_max before its bias test passed";
    case MLMC_ENODEV: return "no usable CUDA device";
    case MLMC_ECOMM: return "the all-reduce hook failed or another rank reported an error";
    default: return "unknown status";
  }
}

int mlmc_params_default(mlmc_params* p) {
  if (!p) return MLMC_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->u_star = 0.2;
  p->f_coriolis = 1e-4;
  p->H = 600.0;
  p->kappa_sigma = 1.3;
  p->kappa_tau = 0.5;
  p->c_f = 15.0;
  p->eps_reg_frac = 1e-3;
  p->z0 = 60.0;
  p->w0 = 0.0;
  p->T = 600.0;
  p->qoi_threshold = 60.0;
  p->w0_mode = 1;
  p->M0 = 8;
  p->level_min = 0;
  p->L_max = 10;
  p->coupling = 0;
  p->drift_outside = 0;
  p->n_init = 10000;
  p->precision = MLMC_FP32;
  p->stream_id = 0;
  p->allow_unstable = 0;
  p->qoi1_mode = 0;
  p->smooth_r = 4;
  p->qoi_a = 0.0;
  p->qoi_b = 0.0;
  p->smooth_delta = 0.0;
  return MLMC_OK;
}

int mlmc_set_tuning(int integrator, int precision, int variant, int items_per_block,
                    int blocks_per_sm) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (precision != MLMC_FP32 && precision != MLMC_FP64) return MLMC_EINVAL;
  if (variant != 1 && variant != 3 && variant != 4 && variant != 12 && variant != 13)
    return MLMC_EINVAL;
  if (precision == MLMC_FP64 && variant != 1) return MLMC_EINVAL;
  if (items_per_block < 1 || items_per_block > 1024) return MLMC_EINVAL;
  if (blocks_per_sm < 0 || blocks_per_sm > kMaxBlocksPerSM) return MLMC_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[integrator][precision] = Tune{variant, items_per_block, blocks_per_sm};
  return MLMC_OK;
}

int mlmc_get_tuning(int integrator, int precision, int32_t out[3]) {
  if (!out || integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (precision != MLMC_FP32 && precision != MLMC_FP64) return MLMC_EINVAL;
  const Tune t = tune_of(precision, integrator);
  out[0] = t.variant;
  out[1] = t.items_per_block;
  out[2] = t.blocks_per_sm;
  return MLMC_OK;
}

int mlmc_device_info(int32_t out[3]) {
  if (!out) return MLMC_EINVAL;
  DevInfo di;
  int rc = device_info(&di);
  if (rc != MLMC_OK) return rc;
  out[0] = di.sms;
  out[1] = di.cc;
  out[2] = 1;
  return MLMC_OK;
}

int mlmc_stable_level_min(const mlmc_params* p, int integrator, int32_t* level) {
  if (!level || integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, 0, &hm);
  if (rc) return rc;
  *level = 0;
  if (integrator != MLMC_SE) return MLMC_OK;
  const double lam = lambda_max(hm);
  for (int l = 0; l <= 40; ++l) {
    if (lam * (p->T / (double)((int64_t)p->M0 << l)) < 2.0) {
      *level = l;
      return MLMC_OK;
    }
  }
  return MLMC_EINVAL;
}

size_t mlmc_workspace_bytes(const mlmc_params* p, int max_requests) {
  (void)p;
  (void)max_requests;
  return workspace_needed();
}

int mlmc_level_sums(int level, uint64_t N, int integrator, const mlmc_params* p, uint64_t seed,
                    uint64_t path_offset, void* workspace, size_t ws_bytes, void* stream,
                    mlmc_level_result* out) {
  NvtxRange nvtx_range("mlmc_level_sums");
  if (!out || integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  Workspace w;
  if ((rc = carve(workspace, ws_bytes, &w))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = p->precision;
  const int grid = hm.adapt ? grid_adapt(prec, integrator, N) : grid_for(prec, integrator, false, N);
  if (grid <= 0) return MLMC_ENODEV;
  if (N > (uint64_t)grid * kBlock * 0x7FFFFFFFull) return MLMC_EINVAL;  // per-thread counters
  rc = cuda_status(launch_level_sums(prec, integrator, hm, ls, N, path_offset, w.partials, grid, st));
  if (rc) return rc;
  rc = cuda_status(launch_finalize(w.partials, grid, fixed_steps(hm, ls, N), w.results, st));
  if (rc) return rc;
  rc = cuda_status(cudaMemcpyAsync(out, w.results, sizeof(*out), cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = cuda_status(cudaStreamSynchronize(st));
  if (rc) return rc;
  return out->n_nonfinite ? MLMC_ENONFINITE : MLMC_OK;
}

// Work items per resident block of an adaptive launch (its pairs' costs vary,
// so the tuned uniform kernel's item size does not carry over).
static constexpr int kAdaptItemsPerBlock = 4;

// Plan a multi-level launch: requests sorted by per-pair cost (finest level
// first), split into items of about total / (items_per_block * grid)
// path-steps, each a whole number of block passes over its pairs; the item
// size doubles until the plan has at most max_items items.  Items are capped
// below 2^31 pairs (in whole passes); a batch that still needs more than
// max_items items returns too_many_rc.  On a packed kernel, a request whose
// pairs are long against a thread's share of the launch runs one pair per
// thread (single).
// Both batched forms (workspace and allocation-free) plan with this
// function, so a batch that fits both gets the same items.
static int plan_requests(const HostModel& hm, const mlmc_level_request* reqs, int n_req, int integ,
                         const mlmc_params* p, int grid, uint32_t max_items, int too_many_rc,
                         ReqPlan* plan, int* order, uint32_t* n_items_out) {
  if (!reqs || n_req < 1 || n_req > kMaxReq) return MLMC_EINVAL;
  double total = 0.0;
  for (int r = 0; r < n_req; ++r) {
    LevelSpec ls;
    int rc = level_spec(hm, reqs[r].level, &ls);
    if (rc) return rc;
    if ((rc = check_stable(integ, p, hm, ls))) return rc;
    total += (double)reqs[r].count * (double)steps_per_pair(ls);
  }
  for (int r = 0; r < n_req; ++r) order[r] = r;
  // insertion sort by level, finest first (stable)
  for (int i = 1; i < n_req; ++i) {
    int v = order[i], j = i - 1;
    while (j >= 0 && reqs[order[j]].level < reqs[v].level) { order[j + 1] = order[j]; --j; }
    order[j + 1] = v;
  }
  // about items_per_block items per resident block
  const int ipb = hm.adapt ? kAdaptItemsPerBlock : items_per_block(p->precision, integ);
  double target = total / ((double)ipb * (double)grid);
  if (target < 1.0) target = 1.0;
  // the adaptive kernels run one pair per thread at a time
  const uint64_t lane_paths = hm.adapt ? (uint64_t)kBlock : min_item_paths(p->precision, integ);
  const bool packed = lane_paths > (uint64_t)kBlock;
  // requests whose pairs are long against a thread's share run one pair per thread
  const double single_steps = kSingleShare * total / ((double)grid * (double)kBlock);
  for (int pass = 0; pass < 64; ++pass) {
    uint64_t items = 0;
    bool capped = false;
    for (int k = 0; k < n_req; ++k) {
      const mlmc_level_request& q = reqs[order[k]];
      LevelSpec ls;
      level_spec(hm, q.level, &ls);
      const bool single = packed && (double)steps_per_pair(ls) >= single_steps;
      const uint64_t min_paths = single ? (uint64_t)kBlock : lane_paths;
      double ppi = std::floor(target / (double)steps_per_pair(ls));
      uint64_t item_paths = ppi < (double)min_paths ? min_paths : (uint64_t)ppi;
      item_paths -= item_paths % min_paths;   // whole passes of the block over its pairs
      if (item_paths > 0x7FFFFFFFull) {   // at most 2^31 - 1 pairs, in whole passes
        item_paths = 0x7FFFFFFFull - 0x7FFFFFFFull % min_paths;
        capped = true;
      }
      const uint64_t n_it = q.count ? (q.count + item_paths - 1) / item_paths : 0;
      plan[k].lv = ls;
      plan[k].first = q.first;
      plan[k].count = q.count;
      plan[k].item_paths = (uint32_t)item_paths;
      plan[k].n_items = (uint32_t)n_it;
      plan[k].item_base = (uint32_t)items;
      plan[k].single = single ? 1u : 0u;
      plan[k].path_steps = fixed_steps(hm, ls, q.count);
      items += n_it;
    }
    if (items <= (uint64_t)max_items) {
      *n_items_out = (uint32_t)items;
      return MLMC_OK;
    }
    if (capped) break;
    target *= 2.0;
  }
  return too_many_rc;
}

static int multilevel_launch(const mlmc_level_request* reqs, int n_req, int integrator,
                             const mlmc_params* p, uint64_t seed, void* workspace, size_t ws_bytes,
                             cudaStream_t st, mlmc_level_result* d_sorted, ReqPlan* plan,
                             int* order) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  Workspace w;
  if ((rc = carve(workspace, ws_bytes, &w))) return rc;
  const int prec = p->precision;
  const int grid = hm.adapt ? grid_adapt_multi(prec, integrator) : grid_for(prec, integrator, true, 0);
  if (grid <= 0) return MLMC_ENODEV;
  uint32_t n_items = 0;
  if ((rc = plan_requests(hm, reqs, n_req, integrator, p, grid, (uint32_t)kMaxItems, MLMC_EINVAL,
                          plan, order, &n_items)))
    return rc;
  rc = cuda_status(cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), st));
  if (rc) return rc;
  rc = cuda_status(launch_multilevel(prec, integrator, hm, plan, n_req, n_items, w.partials,
                                     w.counter, grid, st));
  if (rc) return rc;
  return cuda_status(launch_finalize_multi(w.partials, plan, n_req, d_sorted, st));
}

int mlmc_multilevel_plan(const mlmc_level_request* reqs, int n_req, int integrator,
                         const mlmc_params* p, int grid, uint32_t* out) {
  if (!out || !reqs || n_req < 1 || n_req > kMaxReq || grid < 1) return MLMC_EINVAL;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, 0, &hm);
  if (rc) return rc;
  ReqPlan plan[kMaxReq];
  int order[kMaxReq];
  uint32_t n_items = 0;
  if ((rc = plan_requests(hm, reqs, n_req, integrator, p, grid, (uint32_t)kMaxItems, MLMC_EINVAL,
                          plan, order, &n_items)))
    return rc;
  for (int k = 0; k < n_req; ++k) {
    out[5 * k + 0] = (uint32_t)order[k];
    out[5 * k + 1] = plan[k].item_paths;
    out[5 * k + 2] = plan[k].n_items;
    out[5 * k + 3] = plan[k].item_base;
    out[5 * k + 4] = plan[k].single;
  }
  return MLMC_OK;
}

int mlmc_multilevel_sums_async(const mlmc_level_request* reqs, int n_req, int integrator,
                               const mlmc_params* p, uint64_t seed, void* workspace,
                               size_t ws_bytes, void* stream, mlmc_level_result* d_out) {
  NvtxRange nvtx_range("mlmc_multilevel_sums");
  if (!d_out || !reqs || n_req < 1 || n_req > kMaxReq) return MLMC_EINVAL;
  // requests must already be in non-increasing level order so that d_out
  // lines up with reqs (the async form cannot permute on the device for free)
  for (int r = 1; r < n_req; ++r)
    if (reqs[r].level > reqs[r - 1].level) return MLMC_EINVAL;
  ReqPlan plan[kMaxReq];
  int order[kMaxReq];
  return multilevel_launch(reqs, n_req, integrator, p, seed, workspace, ws_bytes,
                           (cudaStream_t)stream, d_out, plan, order);
}

int mlmc_multilevel_sums(const mlmc_level_request* reqs, int n_req, int integrator,
                         const mlmc_params* p, uint64_t seed, void* workspace, size_t ws_bytes,
                         void* stream, mlmc_level_result* out) {
  if (!out || !reqs || n_req < 1 || n_req > kMaxReq) return MLMC_EINVAL;
  ReqPlan plan[kMaxReq];
  int order[kMaxReq];
  Workspace w;
  int rc = carve(workspace, ws_bytes, &w);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = multilevel_launch(reqs, n_req, integrator, p, seed, workspace, ws_bytes, st, w.results,
                         plan, order);
  if (rc) return rc;
  mlmc_level_result tmp[kMaxReq];
  rc = cuda_status(cudaMemcpyAsync(tmp, w.results, sizeof(mlmc_level_result) * n_req,
                                   cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = cuda_status(cudaStreamSynchronize(st));
  if (rc) return rc;
  uint64_t bad = 0;
  for (int k = 0; k < n_req; ++k) {
    out[order[k]] = tmp[k];
    bad += tmp[k].n_nonfinite;
  }
  return bad ? MLMC_ENONFINITE : MLMC_OK;
}

// Adaptive MLMC (Giles 2008, Section 5; the rule the paper cites for N_l):
//   1. L = level_min;  2. n_init samples on level L;  3. N_l = ceil(2 eps^-2
//   sqrt(V_l / C_l) sum_k sqrt(V_k C_k));  4. run the extra samples;
//   5. if L >= level_min + 2 stop when max(|Yhat_{L-1}| / 2, |Yhat_L|) <
//   eps / sqrt(2);  6. else L += 1 (up to L_max) and go to 2.
// Each pass of steps 2 and 4 is one batched multi-level launch.
//
// Sharded form (one rank per GPU): each pass,
// rank r of W integrates its contiguous slice of every level's new path
// range, the per-level sums (count, diverged, steps, the twelve FP64 sums and
// an error flag) are summed over the ranks by the caller's all-reduce, and
// every rank then takes the same N_l and bias-test decisions from the same
// totals.  W = 1 without a reduce hook is mlmc_estimate.
struct Shard {
  int rank, world;
  mlmc_allreduce_fn reduce;
  void* ctx;
};
constexpr int kShardWidth = 16;  // doubles per level in the reduced buffer

// The host-driven estimate is a state machine over mlmc_estimate_state:
// phase 0 runs the new level's n_init samples, phase 1 the top-up of every
// level to Eq. 12's N_l and then the bias test (Eq. 11), which either ends
// the estimate or adds a level.  Each pass is one multi-level launch over
// this rank's contiguous slice of every level's new path range, followed by
// the all-reduce of the sharded form; the state changes only when the pass
// succeeded on every rank.
static int estimate_pass_impl(mlmc_estimate_state* st, const mlmc_params* p, void* workspace,
                              size_t ws_bytes, void* stream, const Shard& sh) {
  NvtxRange nvtx_range("mlmc_estimate pass");
  if (!st || !p) return MLMC_EINVAL;
  if (st->phase == 2) return 1;
  if (st->phase != 0 && st->phase != 1) return MLMC_EINVAL;
  const int lmin = p->level_min, L = st->L;
  if (L < lmin || L > p->L_max || L >= MLMC_MAX_LEVELS) return MLMC_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  const double eps = st->eps;
  uint64_t dN[MLMC_MAX_LEVELS] = {0};
  if (st->phase == 0) {
    dN[L] = (uint64_t)p->n_init;
  } else {
    double V[MLMC_MAX_LEVELS] = {0}, Cl[MLMC_MAX_LEVELS] = {0}, total = 0.0;
    for (int l = lmin; l <= L; ++l) {
      const double n = (double)st->n[l];
      const double m1 = st->sum[l][0][0], m2 = st->sum[l][0][1];
      V[l] = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      if (V[l] < 0.0) V[l] = 0.0;
      // C_l: integrator steps of one sample, M + M/2 with uniform timesteps
      // (M on level_min) and the counted mean with adaptive ones
      Cl[l] = (double)st->path_steps[l] / (double)(st->n[l] + st->n_nonfinite[l]);
      total += std::sqrt(V[l] * Cl[l]);
    }
    for (int l = lmin; l <= L; ++l) {
      const double Nopt = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / Cl[l]) * total);
      dN[l] = Nopt > (double)st->n_done[l] ? (uint64_t)(Nopt - (double)st->n_done[l]) : 0;
    }
  }
  double buf[MLMC_MAX_LEVELS * kShardWidth];
  int err = MLMC_OK;
  mlmc_level_request rq[MLMC_MAX_LEVELS];
  int nrq = 0;
  for (int l = lmin; l <= L; ++l) {
    double* b = buf + (l - lmin) * kShardWidth;
    for (int k = 0; k < kShardWidth; ++k) b[k] = 0.0;
    if (!dN[l]) continue;
    const uint64_t share = dN[l] / (uint64_t)sh.world, rem = dN[l] % (uint64_t)sh.world;
    const uint64_t r_ = (uint64_t)sh.rank;
    const uint64_t cnt = share + (r_ < rem ? 1 : 0);
    const uint64_t first = st->n_done[l] + r_ * share + (r_ < rem ? r_ : rem);
    if (!cnt) continue;
    rq[nrq].level = l;
    rq[nrq].reserved = 0;
    rq[nrq].first = first;
    rq[nrq].count = cnt;
    ++nrq;
  }
  if (nrq) {
    mlmc_level_result res[MLMC_MAX_LEVELS];
    int rc = mlmc_multilevel_sums(rq, nrq, st->integrator, p, st->seed, workspace, ws_bytes,
                                  stream, res);
    if (rc && rc != MLMC_ENONFINITE) err = rc;
    for (int k = 0; k < nrq && !err; ++k) {
      double* b = buf + (rq[k].level - lmin) * kShardWidth;
      b[0] = (double)res[k].n;
      b[1] = (double)res[k].n_nonfinite;
      b[2] = (double)res[k].path_steps;
      for (int q = 0; q < 2; ++q)
        for (int j = 0; j < 6; ++j) b[3 + 6 * q + j] = res[k].sum[q][j];
    }
  }
  const int nl = L - lmin + 1;
  buf[nl * kShardWidth - 1] = err ? 1.0 : 0.0;   // last slot of the last level: error flag
  if (sh.world > 1) {
    if (sh.reduce(buf, nl * kShardWidth, sh.ctx) != 0) return MLMC_ECOMM;
  }
  if (buf[nl * kShardWidth - 1] != 0.0) return err ? err : MLMC_ECOMM;  // a rank failed
  for (int l = lmin; l <= L; ++l) {
    const double* b = buf + (l - lmin) * kShardWidth;
    if (!dN[l]) continue;
    st->n[l] += (uint64_t)b[0];
    st->n_nonfinite[l] += (uint64_t)b[1];
    st->path_steps[l] += (uint64_t)b[2];
    for (int q = 0; q < 2; ++q)
      for (int k = 0; k < 6; ++k) st->sum[l][q][k] += b[3 + 6 * q + k];
    st->n_done[l] += dN[l];
  }
  if (st->phase == 0) {
    st->phase = 1;
  } else {
    bool conv = false;
    if (L >= lmin + 2) {
      const double yL = std::fabs(st->sum[L][0][0] / (double)st->n[L]);
      const double yL1 = std::fabs(st->sum[L - 1][0][0] / (double)st->n[L - 1]);
      conv = std::fmax(yL1 / 2.0, yL) < eps / std::sqrt(2.0);
    }
    if (conv || L >= p->L_max) {
      st->converged = conv ? 1 : 0;
      st->phase = 2;
    } else {
      st->L = L + 1;
      st->phase = 0;
    }
  }
  st->passes += 1;
  st->seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st->phase == 2 ? 1 : MLMC_OK;
}

static int estimate_result_impl(const mlmc_estimate_state* st, const mlmc_params* p,
                                mlmc_result* out) {
  if (!st || !p || !out) return MLMC_EINVAL;
  const int lmin = p->level_min, L = st->L;
  if (L < lmin || L >= MLMC_MAX_LEVELS) return MLMC_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->L = L;
  out->converged = st->converged;
  for (int q = 0; q < 2; ++q) {
    double est = 0.0, var = 0.0;
    for (int l = lmin; l <= L; ++l) {
      const double n = (double)st->n[l];
      const double m1 = st->sum[l][q][0], m2 = st->sum[l][q][1];
      est += m1 / n;
      const double v = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      var += (v > 0.0 ? v : 0.0) / n;
    }
    out->estimate[q] = est;
    out->est_variance[q] = var;
  }
  bool nonfinite = false;
  for (int l = lmin; l <= L; ++l) {
    const double n = (double)st->n[l];
    out->N[l] = st->n[l];
    out->mean_y[l] = st->sum[l][0][0] / n;
    const double v =
        n > 1.0 ? (st->sum[l][0][1] - st->sum[l][0][0] * st->sum[l][0][0] / n) / (n - 1.0) : 0.0;
    out->V[l] = v > 0.0 ? v : 0.0;
    out->total_path_steps += st->path_steps[l];
    out->n_nonfinite += st->n_nonfinite[l];
    nonfinite |= st->n_nonfinite[l] > 0;
  }
  out->seconds = st->seconds;
  if (nonfinite) return MLMC_ENONFINITE;
  return st->converged ? MLMC_OK : MLMC_ENOTCONV;
}

static int estimate_impl(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                         void* workspace, size_t ws_bytes, void* stream, mlmc_result* out,
                         const Shard& sh) {
  if (!out) return MLMC_EINVAL;
  if (sh.world < 1 || sh.rank < 0 || sh.rank >= sh.world || (sh.world > 1 && !sh.reduce))
    return MLMC_EINVAL;
  mlmc_estimate_state st;
  int rc = mlmc_estimate_begin(eps, integrator, p, seed, &st);
  while (rc == MLMC_OK) rc = estimate_pass_impl(&st, p, workspace, ws_bytes, stream, sh);
  if (rc != 1) return rc;
  return estimate_result_impl(&st, p, out);
}

int mlmc_estimate_begin(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                        mlmc_estimate_state* st) {
  if (!st || !p || !(eps > 0.0)) return MLMC_EINVAL;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (p->L_max < p->level_min + 2 || p->L_max >= MLMC_MAX_LEVELS || p->n_init < 2 ||
      p->level_min < 0)
    return MLMC_EINVAL;
  std::memset(st, 0, sizeof(*st));
  st->eps = eps;
  st->seed = seed;
  st->integrator = integrator;
  st->L = p->level_min;
  st->phase = 0;
  return MLMC_OK;
}

int mlmc_estimate_pass(mlmc_estimate_state* st, const mlmc_params* p, void* workspace,
                       size_t ws_bytes, void* stream) {
  return estimate_pass_impl(st, p, workspace, ws_bytes, stream, Shard{0, 1, nullptr, nullptr});
}

int mlmc_estimate_result(const mlmc_estimate_state* st, const mlmc_params* p, mlmc_result* out) {
  return estimate_result_impl(st, p, out);
}

int mlmc_estimate(double eps, int integrator, const mlmc_params* p, uint64_t seed, void* workspace,
                  size_t ws_bytes, void* stream, mlmc_result* out) {
  return estimate_impl(eps, integrator, p, seed, workspace, ws_bytes, stream, out,
                       Shard{0, 1, nullptr, nullptr});
}

int mlmc_estimate_sharded(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                          int rank, int world, mlmc_allreduce_fn reduce, void* ctx,
                          void* workspace, size_t ws_bytes, void* stream, mlmc_result* out) {
  return estimate_impl(eps, integrator, p, seed, workspace, ws_bytes, stream, out,
                       Shard{rank, world, reduce, ctx});
}

// Plain Monte Carlo (Eq. StMCestimator) at one timestep: a pilot run sets
// N = ceil(2 Var[P] / eps^2) (variance part of Eq. StMCerror at eps^2 / 2).
int mlmc_stmc_estimate(double eps, int level, int n_pilot, int integrator, const mlmc_params* p,
                       uint64_t seed, void* workspace, size_t ws_bytes, void* stream,
                       mlmc_result* out) {
  if (!out || !p || !(eps > 0.0) || n_pilot < 2) return MLMC_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  mlmc_params q = *p;
  q.level_min = level;  // plain paths on this level
  mlmc_level_result a, b;
  int status = MLMC_OK;
  int rc = mlmc_level_sums(level, (uint64_t)n_pilot, integrator, &q, seed, 0, workspace, ws_bytes,
                           stream, &a);
  if (rc == MLMC_ENONFINITE) status = rc;
  else if (rc) return rc;
  const double n = (double)a.n;
  double var = n > 1.0 ? (a.sum[0][1] - a.sum[0][0] * a.sum[0][0] / n) / (n - 1.0) : 0.0;
  if (var < 0.0) var = 0.0;
  const double Nt = std::ceil(2.0 * var / (eps * eps));
  uint64_t extra = Nt > (double)n_pilot ? (uint64_t)(Nt - (double)n_pilot) : 0;
  std::memset(&b, 0, sizeof(b));
  if (extra) {
    rc = mlmc_level_sums(level, extra, integrator, &q, seed, (uint64_t)n_pilot, workspace, ws_bytes,
                         stream, &b);
    if (rc == MLMC_ENONFINITE) status = rc;
    else if (rc) return rc;
  }
  std::memset(out, 0, sizeof(*out));
  const double nt = (double)(a.n + b.n);
  for (int qq = 0; qq < 2; ++qq) {
    const double m1 = a.sum[qq][0] + b.sum[qq][0], m2 = a.sum[qq][1] + b.sum[qq][1];
    out->estimate[qq] = m1 / nt;
    const double v = nt > 1.0 ? (m2 - m1 * m1 / nt) / (nt - 1.0) : 0.0;
    out->est_variance[qq] = (v > 0.0 ? v : 0.0) / nt;
  }
  out->L = level;
  out->converged = 1;
  out->N[level] = a.n + b.n;
  out->V[level] = var;
  out->mean_y[level] = out->estimate[0];
  out->total_path_steps = a.path_steps + b.path_steps;
  out->n_nonfinite = a.n_nonfinite + b.n_nonfinite;
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}

int mlmc_level_paths_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                           uint64_t seed, uint64_t path_offset, void* d_states, int32_t* d_flags,
                           void* stream) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (N && (!d_states || !d_flags)) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  return cuda_status(launch_paths(p->precision, integrator, hm, ls, N, path_offset, d_states,
                                  d_flags, (cudaStream_t)stream));
}

int mlmc_level_paths_variant_async(int variant, int level, uint64_t N, int integrator,
                                   const mlmc_params* p, uint64_t seed, uint64_t path_offset,
                                   void* d_states, int32_t* d_flags, void* stream) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (variant != 0 && variant != 1 && variant != 3 && variant != 4 && variant != 12 &&
      variant != 13)
    return MLMC_EINVAL;
  if (N && (!d_states || !d_flags)) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (p->precision == MLMC_FP64 && variant > 1) return MLMC_EINVAL;
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (hm.adapt) {   // one adaptive kernel serves every variant
    return cuda_status(launch_adapt_paths(p->precision, integrator, hm, ls, N, path_offset,
                                          d_states, d_flags, nullptr, st));
  }
  return cuda_status(launch_paths_variant(variant, p->precision, integrator, hm, ls, N,
                                          path_offset, d_states, d_flags, st));
}

int mlmc_level_paths_steps_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                                 uint64_t seed, uint64_t path_offset, void* d_states,
                                 int32_t* d_flags, int64_t* d_steps, void* stream) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (N && (!d_states || !d_flags || !d_steps)) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (!hm.adapt) return MLMC_EINVAL;
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  return cuda_status(launch_adapt_paths(p->precision, integrator, hm, ls, N, path_offset, d_states,
                                        d_flags, d_steps, (cudaStream_t)stream));
}

int mlmc_fp32_peak_probe(int iters, void* d_scratch, void* stream, double* flops_per_s) {
  if (iters < 1 || !d_scratch || !flops_per_s) return MLMC_EINVAL;
  DevInfo di;
  int rc = device_info(&di);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = di.sms * kMaxBlocksPerSM;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MLMC_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MLMC_ECUDA; }
  k_ffma_probe<<<grid, kBlock, 0, st>>>((float*)d_scratch, iters);  // warm-up
  cudaEventRecord(e0, st);
  k_ffma_probe<<<grid, kBlock, 0, st>>>((float*)d_scratch, iters);
  cudaEventRecord(e1, st);
  rc = cuda_status(cudaGetLastError());
  if (!rc) rc = cuda_status(cudaEventSynchronize(e1));
  float ms = 0.f;
  if (!rc) rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double flops = 2.0 * 8.0 * 16.0 * (double)iters * (double)grid * kBlock;
  *flops_per_s = flops / (ms * 1e-3);
  return MLMC_OK;
}

int mlmc_path_trace_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                          uint64_t seed, uint64_t path_offset, void* d_trace_f, void* d_trace_c,
                          void* stream) {
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (N && !d_trace_f) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (hm.adapt) return MLMC_EINVAL;  // adaptive paths have no fixed time points
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  return cuda_status(launch_trace(p->precision, integrator, hm, ls, N, path_offset, d_trace_f,
                                  d_trace_c, nullptr, nullptr, (cudaStream_t)stream));
}

int mlmc_path_trace_half_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                               uint64_t seed, uint64_t path_offset, void* d_half_f,
                               void* d_half_c, void* stream) {
  if (integrator != MLMC_BAOAB) return MLMC_EINVAL;
  if (N && !d_half_f) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (hm.adapt) return MLMC_EINVAL;
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  return cuda_status(launch_trace(p->precision, integrator, hm, ls, N, path_offset, nullptr,
                                  nullptr, d_half_f, d_half_c, (cudaStream_t)stream));
}

}  // extern "C"

// ===========================================================================
// Batched launch without any allocation: the scratch lives in a fixed array
// of device memory that belongs to this library.
// ===========================================================================
namespace mlmc {

// Upper bound on the work items of one call; each item needs one 128-byte
// partial slot, so the array is 256 + 4096 * 128 bytes (about 0.5 MiB).  Every
// GPU that loads the library keeps this array until the process exits.
constexpr int kNoAllocItems = 4096;
static __device__ __align__(256) unsigned char g_noalloc_scratch[256 + kNoAllocItems * sizeof(Partial)];

// Device address of the array, looked up once per CUDA context with that
// context current.  Host code cannot use the symbol itself: on the host it
// names a stand-in, not device memory.  The address belongs to a context
// (the device's primary context, or one the caller made current), so the
// cache is keyed on the context's unique id, which the driver never reuses:
// after cudaDeviceReset, or in another context on the same device, the
// lookup runs again.  The driver calls come through the runtime's entry
// point query, so the library does not link the driver library.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
struct NoallocAddr {
  unsigned long long ctx_id;
  void* ptr;
};
static NoallocAddr g_noalloc_addr[64];
static int g_noalloc_n = 0;
static CtxGetCurrentFn g_ctx_get_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the current context; 0 when none is current yet.  Caller holds g_mu.
static int current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&g_ctx_get_current, 12000,
                                         cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&g_ctx_get_id, 12000,
                                         cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess ||
        !g_ctx_get_current || !g_ctx_get_id) {
      g_ctx_get_current = nullptr;
      g_ctx_get_id = nullptr;
      return MLMC_ENODEV;
    }
  }
  void* ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0) return MLMC_ECUDA;
  *id = 0;
  if (ctx && g_ctx_get_id(ctx, id) != 0) return MLMC_ECUDA;
  return MLMC_OK;
}

static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return MLMC_ENODEV;
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  for (int k = 0; id && k < g_noalloc_n; ++k)
    if (g_noalloc_addr[k].ctx_id == id) {
      *out = g_noalloc_addr[k].ptr;
      return MLMC_OK;
    }
  // set-up: with no context current yet this lookup also creates the
  // device's primary context and makes it current
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MLMC_ECUDA;
  if ((rc = current_context_id(&id))) return rc;
  if (id) {
    if (g_noalloc_n == 64) g_noalloc_n = 0;   // a process with more contexts recycles the table
    g_noalloc_addr[g_noalloc_n++] = NoallocAddr{id, p};
  }
  *out = p;
  return MLMC_OK;
}

}  // namespace mlmc

extern "C" int mlmc_multilevel_sums_noalloc(const mlmc_level_request* reqs, int n_req,
                                            int integrator, const mlmc_params* p, uint64_t seed,
                                            void* stream, mlmc_level_result* d_out) {
  if (!d_out || !reqs || n_req < 1 || n_req > kMaxReq) return MLMC_EINVAL;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  for (int r = 1; r < n_req; ++r)
    if (reqs[r].level > reqs[r - 1].level) return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  const int prec = p->precision;
  const int grid = hm.adapt ? grid_adapt_multi(prec, integrator) : grid_for(prec, integrator, true, 0);
  if (grid <= 0) return MLMC_ENODEV;
  // the workspace form's split (the requests are already finest level first,
  // so the plan's order is theirs); only a batch of more than kNoAllocItems
  // items gets larger items
  ReqPlan plan[kMaxReq];
  int order[kMaxReq];
  uint32_t n_items = 0;
  if ((rc = plan_requests(hm, reqs, n_req, integrator, p, grid, (uint32_t)kNoAllocItems,
                          MLMC_EWORKSPACE, plan, order, &n_items)))
    return rc;
  unsigned int* counter = (unsigned int*)scratch;
  Partial* partials = (Partial*)((char*)scratch + 256);
  cudaStream_t st = (cudaStream_t)stream;
  // the work counter must start at zero; every partial slot the reduction
  // reads is written first by its item, so nothing else needs clearing
  rc = cuda_status(cudaMemsetAsync(counter, 0, sizeof(unsigned int), st));
  if (rc) return rc;
  rc = cuda_status(launch_multilevel(prec, integrator, hm, plan, n_req, n_items, partials, counter,
                                     grid, st));
  if (rc) return rc;
  return cuda_status(launch_finalize_multi(partials, plan, n_req, d_out, st));
}
