// mlmc_serve.cu -- continuous-batching server of dispersion queries.
//
// Each query is one adaptive MLMC estimate (Giles 2008, Section 5, the rule
// the paper adopts in its Section 6) of its own scenario (u*, H, z0, T, eps).
// A query holds a device slot (its Model) while active.  A pass of a query's
// driver (the n_init samples of a new level, or the extra samples its
// variance estimate asks for) is cut into chunks of at most kChunkSteps
// path-steps; every tick the server fills ONE request table with chunks of
// the active queries -- the query with the least work left in its pass
// first, up to kTickSteps path-steps in all -- runs one persistent
// multi-level launch over it, reduces each chunk in item order, folds the
// chunks into their queries in chunk order, and advances a query's driver
// once its pass is complete.  Finished queries release their slot and queued
// queries are admitted in arrival order while a slot is free.  Light queries
// therefore do not wait behind a heavy query's whole pass, and a tick stays
// short however many heavy queries are active.
//
// The chunks of a pass, a chunk's split into work items and the order in
// which chunks are folded depend only on the query (and the server's grid),
// never on what else is active, so a query's sums -- and its estimate -- are
// bitwise the same alone and among other queries; the tick budget decides
// only WHEN a chunk runs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <unordered_map>
#include <vector>

#include "mlmc_internal.h"

namespace mlmc {

constexpr int kMaxTableReq = 2048;          // requests per tick
constexpr double kItemTarget = 1 << 20;     // largest work item, path-steps
constexpr uint64_t kMaxItemsPerReq = 1024;  // items one request may use
constexpr double kChunkSteps = 1 << 26;     // path-steps of one chunk (one request)
constexpr double kTickSteps = 1 << 28;      // path-steps of one tick (at least one chunk)
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
  // Ndone: samples folded; dN: samples of the current pass not yet issued
  uint64_t Ndone[kQLevels] = {0}, dN[kQLevels] = {0};
  int skipped = 0;  // ticks in a row this query waited with work pending
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

struct mlmc_server_s {
  int integ = 0, prec = 0, max_active = 0, grid = 0;
  uint64_t seed = 0;
  cudaStream_t st = nullptr;
  // device memory, carved from the caller's workspace
  unsigned int* d_counter = nullptr;
  char* d_models = nullptr;
  PlanReq* d_reqs = nullptr;
  mlmc_level_result* d_results = nullptr;
  Partial* d_partials = nullptr;
  // pinned host staging
  char* h_models = nullptr;
  PlanReq* h_reqs = nullptr;
  mlmc_level_result* h_results = nullptr;
  bool models_dirty = false;
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Query> q;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;   // admission order
  std::vector<int> free_slots;
  std::vector<uint64_t> done_order;
  // statistics
  uint64_t ticks = 0, path_steps = 0, completed = 0;
  double busy_s = 0.0;
};

static size_t server_bytes(int max_active) {
  return 256 + (size_t)max_active * kModelSlot + (size_t)kMaxTableReq * sizeof(PlanReq) +
         (size_t)kMaxTableReq * sizeof(mlmc_level_result) + (size_t)kMaxItems * sizeof(Partial);
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
  const int grid = grid_for(precision, integrator, true, 0);
  if (grid <= 0) return MLMC_ENODEV;
  mlmc_server_s* s = new mlmc_server_s();
  s->integ = integrator;
  s->prec = precision;
  s->max_active = max_active;
  s->seed = seed;
  s->grid = grid;
  s->st = (cudaStream_t)stream;
  char* b = (char*)workspace;
  s->d_counter = (unsigned int*)b;
  b += 256;
  s->d_models = b;
  b += (size_t)max_active * kModelSlot;
  s->d_reqs = (PlanReq*)b;
  b += (size_t)kMaxTableReq * sizeof(PlanReq);
  s->d_results = (mlmc_level_result*)b;
  b += (size_t)kMaxTableReq * sizeof(mlmc_level_result);
  s->d_partials = (Partial*)b;
  if (cudaHostAlloc((void**)&s->h_models, (size_t)max_active * kModelSlot, cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaHostAlloc((void**)&s->h_reqs, kMaxTableReq * sizeof(PlanReq), cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaHostAlloc((void**)&s->h_results, kMaxTableReq * sizeof(mlmc_level_result),
                    cudaHostAllocDefault) != cudaSuccess) {
    if (s->h_models) cudaFreeHost(s->h_models);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    if (s->h_results) cudaFreeHost(s->h_results);
    delete s;
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

// One scheduling tick: admit, batch, launch, reduce, advance the drivers.
int mlmc_server_tick(mlmc_server s, int* n_done, int* n_active) {
  if (!s) return MLMC_EINVAL;
  const double t0 = now_s();
  int done = 0;
  // admission: a free slot per query, in arrival order
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
    s->models_dirty = true;
    s->active.push_back(qq.id);
  }
  // batch: chunks of the active queries, least pending work first (a
  // query's key halves for every tick it waited, so none waits forever),
  // until the tick's path-step budget, request table or item table is full
  const uint64_t min_item = min_item_paths(s->prec, s->integ);
  std::vector<std::pair<double, size_t>> order;
  for (size_t k = 0; k < s->active.size(); ++k) {
    const Query& qq = s->q[s->active[k]];
    const double w = pending_steps(qq);
    if (w > 0.0) order.push_back({std::ldexp(w, -std::min(qq.skipped, 1000)), k});
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) {
                     return a.first < b.first;
                   });
  std::vector<PlanReq> reqs;
  std::vector<uint64_t> req_query;
  std::vector<uint64_t> in_batch;
  uint64_t items = 0;
  double tick_steps = 0.0;
  bool full = false;
  for (const auto& o : order) {
    Query& qq = s->q[s->active[o.second]];
    bool got = false;
    if (!full) {
      for (int l = qq.L; l >= qq.p.level_min && !full; --l) {
        uint64_t next = qq.Ndone[l];
        while (qq.dN[l] > 0) {
          const uint64_t cp = chunk_paths(qq, l, min_item);
          const uint64_t count = qq.dN[l] < cp ? qq.dN[l] : cp;
          PlanReq r = chunk_request(qq, l, next, count, min_item, s->grid);
          if (!reqs.empty() && (tick_steps + (double)r.path_steps > kTickSteps ||
                                reqs.size() + 1 > (size_t)kMaxTableReq ||
                                items + r.n_items > (uint64_t)kMaxItems)) {
            full = true;
            break;
          }
          r.item_base = (uint32_t)items;
          items += r.n_items;
          tick_steps += (double)r.path_steps;
          reqs.push_back(r);
          req_query.push_back(s->active[o.second]);
          next += count;
          qq.dN[l] -= count;
          got = true;
        }
      }
    }
    if (got) {
      qq.skipped = 0;
      in_batch.push_back(s->active[o.second]);
    } else {
      qq.skipped += 1;
    }
  }
  if (!reqs.empty()) {
    const int n_req = (int)reqs.size();
    std::memcpy(s->h_reqs, reqs.data(), n_req * sizeof(PlanReq));
    cudaStream_t st = s->st;
    int rc = MLMC_OK;
    if (s->models_dirty) {
      rc = cuda_status(cudaMemcpyAsync(s->d_models, s->h_models, (size_t)s->max_active * kModelSlot,
                                       cudaMemcpyHostToDevice, st));
      s->models_dirty = false;
    }
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->d_reqs, s->h_reqs, n_req * sizeof(PlanReq),
                                              cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_status(cudaMemsetAsync(s->d_counter, 0, sizeof(unsigned int), st));
    if (!rc) rc = cuda_status(launch_multilevel_table(s->prec, s->integ, s->d_models, kModelSlot,
                                                      s->d_reqs, n_req, (uint32_t)items,
                                                      s->d_partials, s->d_counter, s->grid, st));
    if (!rc) rc = cuda_status(launch_finalize_table(s->d_partials, s->d_reqs, n_req, s->d_results, st));
    if (!rc) rc = cuda_status(cudaMemcpyAsync(s->h_results, s->d_results,
                                              n_req * sizeof(mlmc_level_result),
                                              cudaMemcpyDeviceToHost, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    if (rc) return rc;
    // fold the chunks into their queries in table order (a query's chunks
    // are contiguous and in issue order)
    for (int k = 0; k < n_req; ++k) {
      Query& qq = s->q[req_query[k]];
      const PlanReq& r = s->h_reqs[k];
      const mlmc_level_result& res = s->h_results[k];
      const int l = r.level;
      for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 6; ++j) qq.S[l][a][j] += res.sum[a][j];
      qq.n[l] += res.n;
      qq.bad[l] += res.n_nonfinite;
      qq.steps[l] += res.path_steps;
      qq.Ndone[l] += r.count;
      s->path_steps += res.path_steps;
    }
    // advance the drivers whose pass is complete
    for (uint64_t id : in_batch) {
      Query& qq = s->q[id];
      if (pending_steps(qq) > 0.0) continue;
      if (q_update(qq)) {
        qq.t_done = now_s();
        q_result(qq);
        qq.state = 2;
        s->free_slots.push_back(qq.slot);
        qq.slot = -1;
        s->done_order.push_back(id);
        ++done;
        ++s->completed;
      }
    }
    std::vector<uint64_t> still;
    for (uint64_t id : s->active)
      if (s->q[id].state == 1) still.push_back(id);
    s->active.swap(still);
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
  if (s->h_models) cudaFreeHost(s->h_models);
  if (s->h_reqs) cudaFreeHost(s->h_reqs);
  if (s->h_results) cudaFreeHost(s->h_results);
  delete s;
  return MLMC_OK;
}

}  // extern "C"
