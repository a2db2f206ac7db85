// mlmc_graph.cu -- the adaptive MLMC loop (Giles 2008, Section 5, the rule
// the paper adopts in its Section 6) run entirely on the device as one CUDA
// graph: an init kernel, then a conditional WHILE node whose body is
//   persistent multi-level kernel -> per-request reduction -> update kernel.
// The update kernel folds the new sums into the per-level totals, applies
// the sample-size rule and the bias test, plans the next launch and sets the
// loop condition; the host only launches the graph and reads the result.
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <nvtx3/nvToolsExt.h>

#include "mlmc_internal.h"

// NVTX ranges name the host-side phases in a profiler's timeline (a no-op
// unless a tool is attached).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace mlmc {

constexpr int kLevels = MLMC_MAX_LEVELS;
constexpr int kMaxIterations = 4 * kLevels;  // default pass limit: more than a converging run takes

// Driver state in the workspace's graph region.  The host reads back the
// leading int32 block only (kGStateHead bytes: done and status).
struct GState {
  int32_t L, pass, iter, converged, status, lmin, Lmax, n_init;
  int32_t M0, grid, done, items_per_block;
  int32_t min_item, max_iter;
  double eps, T;
  uint64_t Ndone[kLevels], dN[kLevels];
  uint64_t n[kLevels], bad[kLevels], steps[kLevels];
  double S[kLevels][2][6];
};

struct GraphRegion {
  GState g;
  DevPlan plan;
  mlmc_result result;
};
static_assert(sizeof(GraphRegion) <= kGraphRegion, "graph region");
constexpr size_t kGStateHead = offsetof(GState, eps);
static_assert(sizeof(GState) % 8 == 0 && sizeof(mlmc_result) % 8 == 0, "zeroed in 8-byte words");

__device__ __forceinline__ uint64_t dev_steps(const GState* g, int l) {
  const int64_t M = (int64_t)g->M0 << l;
  return l > g->lmin ? (uint64_t)(M + M / 2) : (uint64_t)M;
}

// Plan the levels with dN > 0, finest first, exactly as the host planner
// does: items of about total / (items_per_block * grid) path-steps, in
// whole passes of a block over its pairs (at least one); on a packed kernel,
// levels whose pairs are long against a thread's share run one pair per thread.
__device__ void plan_device(const GState* g, DevPlan* plan) {
  double total = 0.0;
  for (int l = g->L; l >= g->lmin; --l)
    if (g->dN[l]) total += (double)g->dN[l] * (double)dev_steps(g, l);
  double target = total / ((double)g->items_per_block * (double)g->grid);
  if (target < 1.0) target = 1.0;
  const bool packed = g->min_item > kBlock;
  const double single_steps = kSingleShare * total / ((double)g->grid * (double)kBlock);
  for (int pass = 0; pass < 40; ++pass) {
    uint64_t items = 0;
    int k = 0;
    for (int l = g->L; l >= g->lmin; --l) {
      if (!g->dN[l]) continue;
      const uint64_t spp = dev_steps(g, l);
      const bool single = packed && (double)spp >= single_steps;
      const uint64_t min_item = single ? (uint64_t)kBlock : (uint64_t)g->min_item;
      const double ppi = floor(target / (double)spp);
      uint64_t item_paths = ppi < (double)min_item ? min_item : (uint64_t)ppi;
      item_paths -= item_paths % min_item;
      if (item_paths > 0x7FFFFFFFull) item_paths = 0x7FFFFFFFull - 0x7FFFFFFFull % min_item;
      const uint64_t n_it = (g->dN[l] + item_paths - 1) / item_paths;
      PlanReq& q = plan->req[k++];
      q.level = l;
      q.coupled = l > g->lmin;
      q.single = single ? 1 : 0;
      q.M = (int64_t)g->M0 << l;
      q.h = g->T / (double)q.M;
      q.first = g->Ndone[l];
      q.count = g->dN[l];
      q.path_steps = g->dN[l] * spp;
      q.item_paths = (uint32_t)item_paths;
      q.n_items = (uint32_t)n_it;
      q.item_base = (uint32_t)items;
      q.slot = 0;
      items += n_it;
    }
    plan->n_req = k;
    plan->n_items = (uint32_t)items;
    if (items <= (uint64_t)kMaxItems) return;
    target *= 2.0;
  }
}

// Zero `bytes` (a multiple of 8) at an 8-byte aligned address, one warp.
__device__ void warp_zero(void* p, size_t bytes, int lane) {
  unsigned long long* q = (unsigned long long*)p;
  for (size_t i = lane; i < bytes / 8; i += 32) q[i] = 0ull;
  __syncwarp();
}

// The result of the loop, by one warp: the per-level terms one lane per
// level, their sums over levels in level order on lane 0.
__device__ void write_result(const GState* g, mlmc_result* out, int lane) {
  __shared__ double s_est[2][kLevels], s_var[2][kLevels];
  const int nl = g->L - g->lmin + 1;
  for (int i = lane; i < nl; i += 32) {
    const int l = g->lmin + i;
    const double n = (double)g->n[l];
    for (int q = 0; q < 2; ++q) {
      const double m1 = g->S[l][q][0], m2 = g->S[l][q][1];
      s_est[q][i] = m1 / n;
      const double v = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      s_var[q][i] = (v > 0.0 ? v : 0.0) / n;
    }
  }
  warp_zero(out, sizeof(*out), lane);
  if (lane == 0) {
    out->L = g->L;
    out->converged = g->converged;
    for (int q = 0; q < 2; ++q) {
      double est = 0.0, var = 0.0;
      for (int i = 0; i < nl; ++i) {
        est += s_est[q][i];
        var += s_var[q][i];
      }
      out->estimate[q] = est;
      out->est_variance[q] = var;
    }
    for (int l = g->lmin; l <= g->L; ++l) {
      out->N[l] = g->n[l];
      out->total_path_steps += g->steps[l];
      out->n_nonfinite += g->bad[l];
    }
  }
  __syncwarp();
  for (int i = lane; i < nl; i += 32) {
    const int l = g->lmin + i;
    const double n = (double)g->n[l];
    out->mean_y[l] = g->S[l][0][0] / n;
    const double v = n > 1.0 ? (g->S[l][0][1] - g->S[l][0][0] * g->S[l][0][0] / n) / (n - 1.0) : 0.0;
    out->V[l] = v > 0.0 ? v : 0.0;
  }
}

__global__ void k_graph_init(GraphRegion* r, unsigned int* counter, int lmin, int Lmax, int n_init,
                             int M0, int grid, int ipb, int min_item, int max_iter, double eps,
                             double T) {
  if (blockIdx.x != 0) return;
  GState* g = &r->g;
  warp_zero(g, sizeof(*g), threadIdx.x);              // the warp clears the state
  if (threadIdx.x != 0) return;
  g->lmin = lmin;
  g->Lmax = Lmax;
  g->n_init = n_init;
  g->M0 = M0;
  g->grid = grid;
  g->items_per_block = ipb;
  g->min_item = min_item;
  g->max_iter = max_iter;
  g->eps = eps;
  g->T = T;
  g->L = lmin;
  g->pass = 0;
  g->dN[lmin] = (uint64_t)n_init;                     // step 2 for the first level
  plan_device(g, &r->plan);
  *counter = 0;
}

// One driver pass after a launch, by one warp.  FP64 instructions are slow
// to issue on this GPU, so the per-request folds and the per-level sample
// sizes go one lane each; sums over levels run in level order, so every
// value is the one a single thread computing level by level gets.
__global__ void k_graph_update(GraphRegion* r, const mlmc_level_result* __restrict__ res,
                               unsigned int* counter, cudaGraphConditionalHandle handle) {
  if (blockIdx.x != 0) return;
  const int lane = threadIdx.x;
  GState* g = &r->g;
  const DevPlan* plan = &r->plan;
  const int n_req = plan->n_req;
  for (int idx = lane; idx < 12 * n_req; idx += 32) {   // fold in the sums just computed
    const int k = idx / 12, j = idx % 12;
    const int l = plan->req[k].level;                  // each level once per plan
    g->S[l][j / 6][j % 6] += res[k].sum[j / 6][j % 6];
  }
  for (int k = lane; k < n_req; k += 32) {
    const int l = plan->req[k].level;
    g->n[l] += res[k].n;
    g->bad[l] += res[k].n_nonfinite;
    g->steps[l] += res[k].path_steps;
    g->Ndone[l] += plan->req[k].count;
    g->dN[l] = 0;
  }
  __syncwarp();
  __shared__ double s_vc[kLevels];
  bool more = false;
  if (g->pass == 0) {                                // step 3: optimal N_l
    const int nl = g->L - g->lmin + 1;
    double V[(kLevels + 31) / 32], C[(kLevels + 31) / 32];
    for (int i = lane, m = 0; i < nl; i += 32, ++m) {
      const int l = g->lmin + i;
      const double n = (double)g->n[l];
      const double m1 = g->S[l][0][0], m2 = g->S[l][0][1];
      V[m] = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      if (V[m] < 0.0) V[m] = 0.0;
      C[m] = (double)dev_steps(g, l);
      s_vc[i] = sqrt(V[m] * C[m]);
    }
    __syncwarp();
    double total = 0.0;
    for (int i = 0; i < nl; ++i) total += s_vc[i];
    bool due = false;
    for (int i = lane, m = 0; i < nl; i += 32, ++m) {
      const int l = g->lmin + i;
      const double Nopt = ceil(2.0 / (g->eps * g->eps) * sqrt(V[m] / C[m]) * total);
      g->dN[l] = Nopt > (double)g->Ndone[l] ? (uint64_t)(Nopt - (double)g->Ndone[l]) : 0;
      due |= g->dN[l] != 0;
    }
    more = __any_sync(0xFFFFFFFFu, due);
    __syncwarp();
    if (lane == 0) g->pass = 1;                      // step 4 runs next if anything is due
    __syncwarp();
  }
  if (lane == 0) {
    g->iter += 1;
    if (!more) {                                     // step 5: bias test
      bool conv = false;
      if (g->L >= g->lmin + 2) {
        const double yL = fabs(g->S[g->L][0][0] / (double)g->n[g->L]);
        const double yL1 = fabs(g->S[g->L - 1][0][0] / (double)g->n[g->L - 1]);
        conv = fmax(yL1 / 2.0, yL) < g->eps / sqrt(2.0);
      }
      if (conv || g->L >= g->Lmax) {
        g->converged = conv ? 1 : 0;
      } else {                                       // step 6: add a level
        g->L += 1;
        g->dN[g->L] = (uint64_t)g->n_init;
        g->pass = 0;
        more = true;
      }
    }
    if (more && g->iter >= g->max_iter) {            // the loop's watchdog
      g->status = MLMC_ETIMEOUT;
      more = false;
    }
    if (more) {
      plan_device(g, &r->plan);
    } else {
      g->done = 1;
    }
    *counter = 0;
    cudaGraphSetConditional(handle, more ? 1u : 0u);
  }
  more = __shfl_sync(0xFFFFFFFFu, more, 0);
  if (!more) {
    __syncwarp();
    write_result(g, &r->result, lane);
  }
}

}  // namespace mlmc

using namespace mlmc;

struct mlmc_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GraphRegion* region = nullptr;
  int lmin = 0;
  // pinned host copies of the result and of the state's leading fields, for
  // graphs launched many times (a pageable copy goes through a staging
  // buffer and takes longer; a one-shot estimate skips the allocation)
  mlmc_result* h_result = nullptr;
  GState* h_head = nullptr;
};

static void graph_free(mlmc_graph_s* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  if (g->e0) cudaEventDestroy(g->e0);
  if (g->e1) cudaEventDestroy(g->e1);
  if (g->h_result) cudaFreeHost(g->h_result);
  if (g->h_head) cudaFreeHost(g->h_head);
  delete g;
}

extern "C" {

static int graph_create(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                        int max_passes, void* workspace, size_t ws_bytes, bool pinned,
                        mlmc_graph* out) {
  if (!out || !p || !(eps > 0.0)) return MLMC_EINVAL;
  *out = nullptr;
  if (max_passes < 0 || max_passes > kMaxIterations) return MLMC_EINVAL;
  if (max_passes == 0) max_passes = kMaxIterations;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (p->L_max < p->level_min + 2 || p->L_max >= MLMC_MAX_LEVELS || p->n_init < 2)
    return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (hm.adapt) return MLMC_EINVAL;  // the device planner assumes fixed steps per pair
  for (int l = p->level_min; l <= p->L_max; ++l) {
    LevelSpec ls;
    if ((rc = level_spec(hm, l, &ls))) return rc;
    if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  }
  Workspace w;
  if ((rc = carve(workspace, ws_bytes, &w))) return rc;
  const int prec = p->precision;
  const int grid = grid_for(prec, integrator, true, 0);
  if (grid <= 0) return MLMC_ENODEV;

  mlmc_graph_s* g = new mlmc_graph_s();
  g->region = (GraphRegion*)w.graph;
  g->lmin = p->level_min;
  cudaGraphNode_t init_node = nullptr;
  size_t n_nodes = 1;
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams cp = {};
  cudaGraph_t body = nullptr;
#define CK(x)                       \
  do {                              \
    if ((x) != cudaSuccess) {       \
      cudaGetLastError();           \
      graph_free(g);                \
      return MLMC_ECUDA;            \
    }                               \
  } while (0)
  CK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  CK(cudaEventCreate(&g->e0));
  CK(cudaEventCreate(&g->e1));
  if (pinned) {
    CK(cudaHostAlloc((void**)&g->h_result, sizeof(mlmc_result), cudaHostAllocDefault));
    CK(cudaHostAlloc((void**)&g->h_head, sizeof(GState), cudaHostAllocDefault));
    // one copy into each now, so that the first launch's read-back is not the first use
    CK(cudaMemcpyAsync(g->h_result, &g->region->result, sizeof(mlmc_result),
                       cudaMemcpyDeviceToHost, g->cap));
    CK(cudaMemcpyAsync(g->h_head, &g->region->g, kGStateHead, cudaMemcpyDeviceToHost, g->cap));
    CK(cudaStreamSynchronize(g->cap));
  }
  CK(cudaGraphCreate(&g->graph, 0));
  // init kernel
  CK(cudaStreamBeginCaptureToGraph(g->cap, g->graph, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  k_graph_init<<<1, 32, 0, g->cap>>>(g->region, w.counter, p->level_min, p->L_max, p->n_init,
                                     p->M0, grid, items_per_block(prec, integrator),
                                     (int)min_item_paths(prec, integrator), max_passes, eps,
                                     p->T);
  CK(cudaGetLastError());
  CK(cudaStreamEndCapture(g->cap, &g->graph));
  CK(cudaGraphGetNodes(g->graph, &init_node, &n_nodes));
  // while (condition) { body }, the condition starts at 1 on every launch
  CK(cudaGraphConditionalHandleCreate(&handle, g->graph, 1, cudaGraphCondAssignDefault));
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond_node;
  CK(cudaGraphAddNode(&cond_node, g->graph, &init_node, nullptr, 1, &cp));
  body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  CK(launch_multilevel_dev(prec, integrator, hm, &g->region->plan, w.partials, w.counter, grid,
                           g->cap));
  CK(launch_finalize_dev(w.partials, &g->region->plan, w.results, g->cap));
  k_graph_update<<<1, 32, 0, g->cap>>>(g->region, w.results, w.counter, handle);
  CK(cudaGetLastError());
  CK(cudaStreamEndCapture(g->cap, &body));
  CK(cudaGraphInstantiate(&g->exec, g->graph, 0));
#undef CK
  *out = g;
  return MLMC_OK;
}

int mlmc_graph_create_ex(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                         int max_passes, void* workspace, size_t ws_bytes, mlmc_graph* out) {
  return graph_create(eps, integrator, p, seed, max_passes, workspace, ws_bytes, true, out);
}

int mlmc_graph_create(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                      void* workspace, size_t ws_bytes, mlmc_graph* out) {
  return graph_create(eps, integrator, p, seed, 0, workspace, ws_bytes, true, out);
}

int mlmc_graph_launch(mlmc_graph g, void* stream) {
  NvtxRange nvtx_range("mlmc_graph_launch");
  if (!g) return MLMC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaEventRecord(g->e0, st) != cudaSuccess) return MLMC_ECUDA;
  if (cudaGraphLaunch(g->exec, st) != cudaSuccess) return MLMC_ECUDA;
  if (cudaEventRecord(g->e1, st) != cudaSuccess) return MLMC_ECUDA;
  return MLMC_OK;
}

int mlmc_graph_result(mlmc_graph g, void* stream, mlmc_result* out) {
  if (!g || !out) return MLMC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  GState head;
  mlmc_result* res = g->h_result ? g->h_result : out;
  GState* hd = g->h_head ? g->h_head : &head;
  if (cudaMemcpyAsync(res, &g->region->result, sizeof(mlmc_result), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(hd, &g->region->g, kGStateHead, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MLMC_ECUDA;
  if (res != out) *out = *res;
  const GState& gs = *hd;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, g->e0, g->e1) == cudaSuccess) out->seconds = 1e-3 * ms;
  if (!gs.done) return MLMC_ECUDA;
  if (gs.status) return gs.status;
  if (out->n_nonfinite) return MLMC_ENONFINITE;
  return out->converged ? MLMC_OK : MLMC_ENOTCONV;
}

int mlmc_graph_destroy(mlmc_graph g) {
  graph_free(g);
  return MLMC_OK;
}

int mlmc_estimate_graph(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                        void* workspace, size_t ws_bytes, void* stream, mlmc_result* out) {
  if (!out) return MLMC_EINVAL;
  mlmc_graph g = nullptr;
  int rc = graph_create(eps, integrator, p, seed, 0, workspace, ws_bytes, false, &g);
  if (rc) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  rc = mlmc_graph_launch(g, stream);
  if (!rc) rc = mlmc_graph_result(g, stream, out);
  if (rc == MLMC_OK || rc == MLMC_ENONFINITE || rc == MLMC_ENOTCONV)
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  mlmc_graph_destroy(g);
  return rc;
}

}  // extern "C"
