// mlmc_serve.cu -- continuous-batching server of dispersion queries.
//
// Each query is one adaptive MLMC estimate (Giles 2008, Section 5, the rule
// the paper adopts in its Section 6) of its own scenario (u*, H, z0, T, eps).
// A query holds a device slot (its Model) while active.  A pass of a query's
// driver (the n_init samples of a new level, or the extra samples its
// variance estimate asks for) is cut into chunks of at most kChunkSteps
// path-steps.  A launch is one persistent multi-level kernel over a request
// table of chunks -- the query with the least work left in its pass first,
// up to kTickSteps path-steps, and only pairs at most kChainRatio times as
// long as the first chunk's (a launch lasts as long as its longest pair) --
// followed by the per-chunk reduction in item order.  Up to kInFlight
// launches run at once, each on its own stream; they are folded in issue
// order, each chunk into its query in chunk order, and a query's driver
// advances once every chunk of its pass is folded.  Finished queries release
// their slot; queued queries take free slots in arrival order.  So a light
// query neither waits for a heavy query's whole pass nor shares a launch
// with its long pairs, and the GPU keeps working on other launches while one
// waits for its longest pair.
//
// The chunks of a pass, a chunk's split into work items and the order in
// which chunks are folded depend only on the query (and the server's grid),
// never on what else is active, so a query's sums -- and its estimate -- are
// bitwise the same alone and among other queries; the scheduling decides
// only WHEN a chunk runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <nvtx3/nvToolsExt.h>
#include <unordered_map>
#include <vector>

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

constexpr int kMaxTableReq = 2048;          // requests per tick
constexpr double kItemTarget = 1 << 20;     // largest work item, path-steps
constexpr uint64_t kMaxItemsPerReq = 1024;  // items one request may use
constexpr double kChunkSteps = 1 << 26;     // path-steps of one chunk (one request)
constexpr double kTickSteps = 1 << 28;      // path-steps of one launch (at least one chunk)
constexpr int kInFlight = 4;                // launches in flight at once
constexpr double kChainRatio = 4.0;         // longest / first pair length in one launch
constexpr double kChainFloor = 2048.0;      // path-steps per pair any launch may hold
constexpr size_t kModelSlot = 512;          // bytes reserved per Model
constexpr int kQLevels = MLMC_MAX_LEVELS;

struct Query {
  uint64_t id = 0;
  mlmc_params p;
  double eps = 0;
  HostModel hm;
  int slot = -1;
  int state = 0;  // 0 queued, 1 active, 2 done
  int L = 0, pass = 0, converged = 0;
  // Ndone: samples folded; Nnext: next sample to issue; dN: samples of the
  // current pass not yet issued
  uint64_t Ndone[kQLevels] = {0}, Nnext[kQLevels] = {0}, dN[kQLevels] = {0};
  int inflight = 0;  // chunks issued and not yet folded
  int skipped = 0;   // launches in a row this query waited with work pending
  uint64_t n[kQLevels] = {0}, bad[kQLevels] = {0}, steps[kQLevels] = {0};
  double S[kQLevels][2][6] = {};
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = MLMC_OK;
  mlmc_result result;
};

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static uint64_t q_steps(const Query& q, int l) {
  const int64_t M = (int64_t)q.p.M0 << l;
  return l > q.p.level_min ? (uint64_t)(M + M / 2) : (uint64_t)M;
}

// Driver update after the query's requests of one tick (same rule as
// mlmc_estimate).  Returns true when the query is finished.
static bool q_update(Query& q) {
  const int lmin = q.p.level_min;
  bool more = false;
  if (q.pass == 0) {
    double V[kQLevels], C[kQLevels], total = 0.0;
    for (int l = lmin; l <= q.L; ++l) {
      const double n = (double)q.n[l];
      const double m1 = q.S[l][0][0], m2 = q.S[l][0][1];
      V[l] = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      if (V[l] < 0.0) V[l] = 0.0;
      C[l] = (double)q_steps(q, l);
      total += std::sqrt(V[l] * C[l]);
    }
    for (int l = lmin; l <= q.L; ++l) {
      const double Nopt = std::ceil(2.0 / (q.eps * q.eps) * std::sqrt(V[l] / C[l]) * total);
      q.dN[l] = Nopt > (double)q.Ndone[l] ? (uint64_t)(Nopt - (double)q.Ndone[l]) : 0;
      more |= q.dN[l] != 0;
    }
    q.pass = 1;
  }
  if (more) return false;
  bool conv = false;
  if (q.L >= lmin + 2) {
    const double yL = std::fabs(q.S[q.L][0][0] / (double)q.n[q.L]);
    const double yL1 = std::fabs(q.S[q.L - 1][0][0] / (double)q.n[q.L - 1]);
    conv = std::fmax(yL1 / 2.0, yL) < q.eps / std::sqrt(2.0);
  }
  if (conv || q.L >= q.p.L_max) {
    q.converged = conv ? 1 : 0;
    return true;
  }
  q.L += 1;
  q.dN[q.L] = (uint64_t)q.p.n_init;
  q.pass = 0;
  return false;
}

static void q_result(Query& q) {
  mlmc_result& out = q.result;
  std::memset(&out, 0, sizeof(out));
  const int lmin = q.p.level_min;
  out.L = q.L;
  out.converged = q.converged;
  for (int k = 0; k < 2; ++k) {
    double est = 0.0, var = 0.0;
    for (int l = lmin; l <= q.L; ++l) {
      const double n = (double)q.n[l];
      const double m1 = q.S[l][k][0], m2 = q.S[l][k][1];
      est += m1 / n;
      const double v = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      var += (v > 0.0 ? v : 0.0) / n;
    }
    out.estimate[k] = est;
    out.est_variance[k] = var;
  }
  for (int l = lmin; l <= q.L; ++l) {
    const double n = (double)q.n[l];
    out.N[l] = q.n[l];
    out.mean_y[l] = q.S[l][0][0] / n;
    const double v = n > 1.0 ? (q.S[l][0][1] - q.S[l][0][0] * q.S[l][0][0] / n) / (n - 1.0) : 0.0;
    out.V[l] = v > 0.0 ? v : 0.0;
    out.total_path_steps += q.steps[l];
    out.n_nonfinite += q.bad[l];
  }
  out.seconds = q.t_done - q.t_submit;
  q.status = out.n_nonfinite ? MLMC_ENONFINITE : (out.converged ? MLMC_OK : MLMC_ENOTCONV);
}

// Paths of one chunk of level l: kChunkSteps worth, at least one full item.
static uint64_t chunk_paths(const Query& q, int l, uint64_t min_item) {
  const double c = std::floor(kChunkSteps / (double)q_steps(q, l));
  return c < (double)min_item ? min_item : (uint64_t)c;
}

static double pending_steps(const Query& q) {
  double w = 0.0;
  for (int l = q.p.level_min; l <= q.L; ++l) w += (double)q.dN[l] * (double)q_steps(q, l);
  return w;
}

// The request of the chunk of `count` samples starting at `first` on level
// l.  Its items spread the chunk over the grid (so a lone light chunk still
// fills the GPU), with at least min_item and at most kItemTarget path-steps'
// worth of paths each.  Depends only on (query, level, first, count, grid).
static PlanReq chunk_request(const Query& q, int l, uint64_t first, uint64_t count,
                             uint64_t min_item, int grid) {
  const uint64_t spp = q_steps(q, l);
  const double cap_d = std::floor(kItemTarget / (double)spp);
  const uint64_t cap = cap_d < (double)min_item ? min_item : (uint64_t)cap_d;
  const uint64_t want = (count + (uint64_t)grid - 1) / (uint64_t)grid;
  uint64_t item_paths = want < min_item ? min_item : (want > cap ? cap : want);
  const uint64_t min_paths = (count + kMaxItemsPerReq - 1) / kMaxItemsPerReq;
  if (item_paths < min_paths) item_paths = min_paths;
  item_paths += (min_item - item_paths % min_item) % min_item;  // whole passes of the block
  if (item_paths > 0x7FFFFFFFull) item_paths = 0x7FFFFFFFull;
  PlanReq r;
  r.level = l;
  r.coupled = l > q.p.level_min;
  r.M = (int64_t)q.p.M0 << l;
  r.h = q.p.T / (double)r.M;
  r.first = first;
  r.count = count;
  r.path_steps = count * spp;
  r.item_paths = (uint32_t)item_paths;
  r.n_items = (uint32_t)((count + item_paths - 1) / item_paths);
  r.item_base = 0;
  r.slot = (uint32_t)q.slot;
  return r;
}

}  // namespace mlmc

using namespace mlmc;

// One launch in flight: its own stream, request table, partials, results
// and completion event.  Launches complete and are folded in issue order.
struct Flight {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  unsigned int* d_counter = nullptr;
  PlanReq* d_reqs = nullptr;
  mlmc_level_result* d_results = nullptr;
  Partial* d_partials = nullptr;
  PlanReq* h_reqs = nullptr;                 // pinned
  mlmc_level_result* h_results = nullptr;    // pinned
  std::vector<uint64_t> req_query;           // the query of each request
  int n_req = 0;
};

struct mlmc_server_s {
  int integ = 0, prec = 0, max_active = 0, grid = 0;
  uint64_t seed = 0;
  char* d_models = nullptr;                  // carved from the caller's workspace
  char* h_models = nullptr;                  // pinned staging of the Model slots
  cudaStream_t up_st = nullptr;              // Model uploads
  cudaEvent_t up_ev = nullptr;               // after the latest upload
  Flight fl[kInFlight];
  std::deque<int> busy;                      // flights in flight, oldest first
  std::vector<int> idle;
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Query> q;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;              // admission order
  std::vector<uint64_t> to_upload;           // admitted, Model not yet on the device
  std::vector<int> free_slots;
  int failed = MLMC_OK;                      // first CUDA error: the server stops
  // statistics
  uint64_t ticks = 0, path_steps = 0, completed = 0;
  double busy_s = 0.0;
};

static size_t flight_bytes() {
  return 256 + (size_t)kMaxTableReq * sizeof(PlanReq) +
         (size_t)kMaxTableReq * sizeof(mlmc_level_result) + (size_t)kMaxItems * sizeof(Partial);
}

static size_t server_bytes(int max_active) {
  return (size_t)max_active * kModelSlot + (size_t)kInFlight * flight_bytes();
}

static void server_free(mlmc_server_s* s) {
  for (Flight& f : s->fl) {
    if (f.st) cudaStreamSynchronize(f.st);
    if (f.done) cudaEventDestroy(f.done);
    if (f.st) cudaStreamDestroy(f.st);
    if (f.h_reqs) cudaFreeHost(f.h_reqs);
    if (f.h_results) cudaFreeHost(f.h_results);
  }
  if (s->up_st) cudaStreamSynchronize(s->up_st);
  if (s->up_ev) cudaEventDestroy(s->up_ev);
  if (s->up_st) cudaStreamDestroy(s->up_st);
  if (s->h_models) cudaFreeHost(s->h_models);
  delete s;
}

// Retire a finished query: result, statistics, its slot back to the pool.
static void retire(mlmc_server_s* s, Query& qq, int* done) {
  qq.t_done = now_s();
  q_result(qq);
  qq.state = 2;
  s->free_slots.push_back(qq.slot);
  qq.slot = -1;
  ++*done;
  ++s->completed;
}

// Fold the oldest flight (waiting for it when `wait`); false when there is
// none or it has not completed.  Its chunks enter their queries in table
// order, which is each query's chunk order; a query whose pass is then
// complete advances its driver and may finish.
static int fold_oldest(mlmc_server_s* s, bool wait, bool* folded, int* done) {
  *folded = false;
  if (s->busy.empty()) return MLMC_OK;
  Flight& f = s->fl[s->busy.front()];
  if (wait) {
    int rc = cuda_status(cudaEventSynchronize(f.done));
    if (rc) return rc;
  } else {
    const cudaError_t e = cudaEventQuery(f.done);
    if (e == cudaErrorNotReady) return MLMC_OK;
    if (e != cudaSuccess) return MLMC_ECUDA;
  }
  std::vector<uint64_t> touched;
  for (int k = 0; k < f.n_req; ++k) {
    Query& qq = s->q[f.req_query[k]];
    const PlanReq& r = f.h_reqs[k];
    const mlmc_level_result& res = f.h_results[k];
    const int l = r.level;
    for (int a = 0; a < 2; ++a)
      for (int j = 0; j < 6; ++j) qq.S[l][a][j] += res.sum[a][j];
    qq.n[l] += res.n;
    qq.bad[l] += res.n_nonfinite;
    qq.steps[l] += res.path_steps;
    qq.Ndone[l] += r.count;
    qq.inflight -= 1;
    s->path_steps += res.path_steps;
    if (touched.empty() || touched.back() != f.req_query[k]) touched.push_back(f.req_query[k]);
  }
  for (uint64_t id : touched) {
    Query& qq = s->q[id];
    if (qq.state != 1 || qq.inflight || pending_steps(qq) > 0.0) continue;
    if (q_update(qq)) retire(s, qq, done);
  }
  std::vector<uint64_t> still;
  for (uint64_t id : s->active)
    if (s->q[id].state == 1) still.push_back(id);
  s->active.swap(still);
  s->idle.push_back(s->busy.front());
  s->busy.pop_front();
  *folded = true;
  return MLMC_OK;
}

// Queued queries take free slots in arrival order.
static void admit(mlmc_server_s* s) {
  while (!s->queue.empty() && !s->free_slots.empty()) {
    Query& qq = s->q[s->queue.front()];
    s->queue.pop_front();
    qq.slot = s->free_slots.back();
    s->free_slots.pop_back();
    qq.state = 1;
    qq.t_admit = now_s();
    qq.L = qq.p.level_min;
    qq.pass = 0;
    qq.dN[qq.L] = (uint64_t)qq.p.n_init;
    model_image(s->prec, qq.hm, s->h_models + (size_t)qq.slot * kModelSlot);
    s->to_upload.push_back(qq.id);
    s->active.push_back(qq.id);
  }
}

// Fill an idle flight with chunks -- least pending work first (a query's
// key halves for every launch it waited), up to the path-step budget, the
// request table and the item table -- and launch it.  *launched is false
// when no query has work to issue.
static int issue(mlmc_server_s* s, bool* launched) {
  *launched = false;
  if (s->idle.empty()) return MLMC_OK;
  const uint64_t min_item = kBlock;  // one pass of a block: one pair per thread
  std::vector<std::pair<double, size_t>> order;
  for (size_t k = 0; k < s->active.size(); ++k) {
    const Query& qq = s->q[s->active[k]];
    const double w = pending_steps(qq);
    if (w > 0.0) order.push_back({std::ldexp(w, -std::min(qq.skipped, 1000)), k});
  }
  if (order.empty()) return MLMC_OK;
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
                     return a.first < b.first;
                   });
  const int fi = s->idle.back();
  Flight& f = s->fl[fi];
  f.req_query.clear();
  int n_req = 0;
  uint64_t items = 0;
  double steps = 0.0, chain_cap = 0.0;
  bool full = false;
  for (const auto& o : order) {
    Query& qq = s->q[s->active[o.second]];
    bool got = false;
    for (int l = qq.L; l >= qq.p.level_min && !full; --l) {
      // a launch lasts at least as long as its longest pair: keep pairs of
      // very different length apart, so short pairs are not held up
      const double spp = (double)q_steps(qq, l);
      if (n_req == 0) chain_cap = std::max(kChainRatio * spp, kChainFloor);
      if (spp > chain_cap) continue;
      while (qq.dN[l] > 0) {
        const uint64_t cp = chunk_paths(qq, l, min_item);
        const uint64_t count = qq.dN[l] < cp ? qq.dN[l] : cp;
        PlanReq r = chunk_request(qq, l, qq.Nnext[l], count, min_item, s->grid);
        if (n_req > 0 && (steps + (double)r.path_steps > kTickSteps || n_req + 1 > kMaxTableReq ||
                          items + r.n_items > (uint64_t)kMaxItems)) {
          full = true;
          break;
        }
        r.item_base = (uint32_t)items;
        items += r.n_items;
        steps += (double)r.path_steps;
        f.h_reqs[n_req++] = r;
        f.req_query.push_back(qq.id);
        qq.Nnext[l] += count;
        qq.dN[l] -= count;
        qq.inflight += 1;
        got = true;
      }
    }
    qq.skipped = got ? 0 : qq.skipped + 1;
  }
  f.n_req = n_req;
  s->idle.pop_back();
  s->busy.push_back(fi);
  int rc = MLMC_OK;
  // Models of newly admitted queries go up on their own stream; every
  // launch waits for the latest upload.
  if (!s->to_upload.empty()) {
    for (uint64_t id : s->to_upload) {
      const Query& qq = s->q[id];
      if (qq.state != 1) continue;
      const size_t off = (size_t)qq.slot * kModelSlot;
      if (!rc) rc = cuda_status(cudaMemcpyAsync(s->d_models + off, s->h_models + off, kModelSlot,
                                                cudaMemcpyHostToDevice, s->up_st));
    }
    s->to_upload.clear();
    if (!rc) rc = cuda_status(cudaEventRecord(s->up_ev, s->up_st));
  }
  if (!rc) rc = cuda_status(cudaStreamWaitEvent(f.st, s->up_ev, 0));
  if (!rc) rc = cuda_status(cudaMemcpyAsync(f.d_reqs, f.h_reqs, n_req * sizeof(PlanReq),
                                            cudaMemcpyHostToDevice, f.st));
  if (!rc) rc = cuda_status(cudaMemsetAsync(f.d_counter, 0, sizeof(unsigned int), f.st));
  if (!rc) rc = cuda_status(launch_multilevel_table_variant(kServeVariant, s->prec, s->integ,
                                                            s->d_models, kModelSlot, f.d_reqs,
                                                            n_req, (uint32_t)items, f.d_partials,
                                                            f.d_counter, s->grid, f.st));
  if (!rc) rc = cuda_status(launch_finalize_table(f.d_partials, f.d_reqs, n_req, f.d_results, f.st));
  if (!rc) rc = cuda_status(cudaMemcpyAsync(f.h_results, f.d_results,
                                            n_req * sizeof(mlmc_level_result),
                                            cudaMemcpyDeviceToHost, f.st));
  if (!rc) rc = cuda_status(cudaEventRecord(f.done, f.st));
  *launched = rc == MLMC_OK;
  return rc;
}

extern "C" {

size_t mlmc_server_workspace_bytes(int max_active) {
  if (max_active < 1) return 0;
  return server_bytes(max_active);
}

int mlmc_server_create(int integrator, int precision, int max_active, uint64_t seed,
                       void* workspace, size_t ws_bytes, void* stream, mlmc_server* out) {
  if (!out) return MLMC_EINVAL;
  *out = nullptr;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (precision != MLMC_FP32 && precision != MLMC_FP64) return MLMC_EINVAL;
  if (max_active < 1 || max_active > 4096) return MLMC_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < server_bytes(max_active))
    return MLMC_EWORKSPACE;
  if (model_bytes(precision) > kModelSlot) return MLMC_EINVAL;
  const int grid = grid_for_variant(kServeVariant, precision, integrator);
  if (grid <= 0) return MLMC_ENODEV;
  mlmc_server_s* s = new mlmc_server_s();
  s->integ = integrator;
  s->prec = precision;
  s->max_active = max_active;
  s->seed = seed;
  s->grid = grid;
  char* b = (char*)workspace;
  s->d_models = b;
  b += (size_t)max_active * kModelSlot;
  bool ok = cudaHostAlloc((void**)&s->h_models, (size_t)max_active * kModelSlot,
                          cudaHostAllocDefault) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->up_st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->up_ev, cudaEventDisableTiming) == cudaSuccess;
  // work the caller queued on its stream (e.g. clearing the workspace)
  // comes before anything the server launches
  cudaEvent_t start = nullptr;
  ok = ok && cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventRecord(start, (cudaStream_t)stream) == cudaSuccess &&
       cudaStreamWaitEvent(s->up_st, start, 0) == cudaSuccess &&
       cudaEventRecord(s->up_ev, s->up_st) == cudaSuccess;
  for (int k = 0; k < kInFlight && ok; ++k) {
    Flight& f = s->fl[k];
    f.d_counter = (unsigned int*)b;
    b += 256;
    f.d_reqs = (PlanReq*)b;
    b += (size_t)kMaxTableReq * sizeof(PlanReq);
    f.d_results = (mlmc_level_result*)b;
    b += (size_t)kMaxTableReq * sizeof(mlmc_level_result);
    f.d_partials = (Partial*)b;
    b += (size_t)kMaxItems * sizeof(Partial);
    ok = cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaHostAlloc((void**)&f.h_reqs, kMaxTableReq * sizeof(PlanReq), cudaHostAllocDefault) ==
             cudaSuccess &&
         cudaHostAlloc((void**)&f.h_results, kMaxTableReq * sizeof(mlmc_level_result),
                       cudaHostAllocDefault) == cudaSuccess &&
         cudaStreamWaitEvent(f.st, start, 0) == cudaSuccess;
    s->idle.push_back(kInFlight - 1 - k);
  }
  if (start) cudaEventDestroy(start);
  if (!ok) {
    server_free(s);
    return MLMC_ECUDA;
  }
  std::memset(s->h_models, 0, (size_t)max_active * kModelSlot);
  for (int k = max_active - 1; k >= 0; --k) s->free_slots.push_back(k);
  *out = s;
  return MLMC_OK;
}

int mlmc_server_submit(mlmc_server s, const mlmc_params* p, double eps, uint64_t* query_id) {
  if (!s || !p || !query_id || !(eps > 0.0)) return MLMC_EINVAL;
  if (p->precision != s->prec) return MLMC_EINVAL;
  if (p->L_max < p->level_min + 2 || p->L_max >= MLMC_MAX_LEVELS || p->n_init < 2)
    return MLMC_EINVAL;
  Query qq;
  int rc = make_host_model(p, s->seed, &qq.hm);
  if (rc) return rc;
  if (qq.hm.adapt) return MLMC_EINVAL;  // batched queries take uniform timesteps

  for (int l = p->level_min; l <= p->L_max; ++l) {
    LevelSpec ls;
    if ((rc = level_spec(qq.hm, l, &ls))) return rc;
    if ((rc = check_stable(s->integ, p, qq.hm, ls))) return rc;
  }
  qq.id = s->next_id++;
  qq.p = *p;
  qq.eps = eps;
  qq.t_submit = now_s();
  std::memset(&qq.result, 0, sizeof(qq.result));
  s->q.emplace(qq.id, qq);
  s->queue.push_back(qq.id);
  *query_id = qq.id;
  return MLMC_OK;
}

// One scheduling step: fold the completed launches, admit, and put one more
// launch in flight; when every flight is busy, or there is nothing new to
// issue, wait for the oldest launch first.  Each call folds or launches at
// least once while any query is active.
int mlmc_server_tick(mlmc_server s, int* n_done, int* n_active) {
  NvtxRange nvtx_range("mlmc_server_tick");
  if (!s) return MLMC_EINVAL;
  if (s->failed) return s->failed;  // launches in flight may be lost: do not fold them
  const double t0 = now_s();
  int done = 0, rc = MLMC_OK;
  bool folded = true, launched = false;
  while (!rc && folded) rc = fold_oldest(s, false, &folded, &done);
  if (!rc) {
    admit(s);
    if (s->idle.empty()) {
      rc = fold_oldest(s, true, &folded, &done);
      if (!rc) admit(s);
    }
  }
  if (!rc) rc = issue(s, &launched);
  if (!rc && !launched && !s->busy.empty()) {
    rc = fold_oldest(s, true, &folded, &done);
    if (!rc) {
      admit(s);
      rc = issue(s, &launched);
    }
  }
  if (rc) {
    s->failed = rc;
    return rc;
  }
  s->ticks += 1;
  s->busy_s += now_s() - t0;
  if (n_done) *n_done = done;
  if (n_active) *n_active = (int)s->active.size() + (int)s->queue.size();
  return MLMC_OK;
}

int mlmc_server_poll(mlmc_server s, uint64_t query_id, mlmc_result* out, double* latency_s) {
  if (!s || !out) return MLMC_EINVAL;
  auto it = s->q.find(query_id);
  if (it == s->q.end()) return MLMC_EINVAL;
  Query& qq = it->second;
  if (qq.state != 2) return 1;  // not finished yet
  *out = qq.result;
  if (latency_s) *latency_s = qq.t_done - qq.t_submit;
  return qq.status;
}

int mlmc_server_release(mlmc_server s, uint64_t query_id) {
  if (!s) return MLMC_EINVAL;
  auto it = s->q.find(query_id);
  if (it == s->q.end() || it->second.state != 2) return MLMC_EINVAL;
  s->q.erase(it);
  return MLMC_OK;
}

int mlmc_server_stats(mlmc_server s, double out[6]) {
  if (!s || !out) return MLMC_EINVAL;
  out[0] = (double)s->ticks;
  out[1] = (double)s->completed;
  out[2] = (double)s->path_steps;
  out[3] = s->busy_s;
  out[4] = (double)s->active.size();
  out[5] = (double)s->queue.size();
  return MLMC_OK;
}

int mlmc_server_destroy(mlmc_server s) {
  if (!s) return MLMC_OK;
  server_free(s);
  return MLMC_OK;
}

}  // extern "C"
