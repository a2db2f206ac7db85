// mlmc_serve.cu -- continuous-batching server of dispersion queries.
//
// Each query is one adaptive MLMC estimate (Giles 2008, Section 5, the rule
// the paper adopts in its Section 6) of its own scenario (u*, H, z0, T, eps).
// An admitted query owns a record in a pool carved from the caller's
// workspace: its Model and its whole per-level state -- the twelve FP64 sums
// of every level, the pair, diverged and step counts, the samples folded,
// the pass targets and the driver's level, pass and plan.  Admission is by
// memory: a queued query is admitted, in arrival order, when a record of its
// size (which grows with its number of levels) fits in the pool.
//
// A pass of a query's driver (the n_init samples of a new level, or the
// extra samples its variance estimate asks for) is cut into chunks of at
// most kChunkSteps path-steps.  A launch is one persistent multi-level
// kernel over a request table of chunks -- the query with the least work
// left in its pass first, up to kTickSteps path-steps, and only pairs at
// most kChainRatio times as long as the first chunk's (a launch lasts as
// long as its longest pair) -- followed by the per-chunk reduction in item
// order.  Up to kInFlight launches run at once, each on its own stream.  A
// fold kernel on one fold stream, which takes the launches in issue order,
// adds each chunk's sums into its query's record in chunk order; when the
// chunks of a pass are all in, it applies the sample-size rule and the bias
// test on the device and writes the query's next plan (or its final result)
// to a small table the host reads back.  The host keeps only what it needs
// to schedule: each query's samples still to issue, its issue pointers and
// its chunks in flight.
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

constexpr int kMaxTableReq = 2048;          // requests per launch
constexpr double kItemTarget = 1 << 20;     // largest work item, path-steps
constexpr uint64_t kMaxItemsPerReq = 1024;  // items one request may use
constexpr double kChunkSteps = 1 << 26;     // path-steps of one chunk (one request)
constexpr double kTickSteps = 1 << 28;      // path-steps of one launch (at least one chunk)
constexpr int kInFlight = 4;                // launches in flight at once
constexpr double kChainRatio = 4.0;         // longest / first pair length in one launch
constexpr double kChainFloor = 2048.0;      // path-steps per pair any launch may hold
constexpr size_t kModelSlot = 512;          // bytes of the Model at the start of a record
constexpr size_t kRecUnit = 256;            // records start and end on 256-byte boundaries
constexpr int kQLevels = MLMC_MAX_LEVELS;
constexpr int kSizingLevels = 17;           // levels per query that the workspace helper assumes

// The device record of a query, after its Model: a header, then nl entries
// (levels lmin .. lmin + nl - 1) of each per-level array.
struct QHead {
  int32_t lmin, Lmax, nl, n_init;
  int32_t L, pass, done, converged;
  int32_t version, M0, pad0, pad1;
  double eps;
  char pad[256 - 56];
};
static_assert(sizeof(QHead) == 256, "record header");
constexpr size_t kQArrays = 12 + 6;  // S[12] doubles; n, bad, steps, Ndone, target, dN

static size_t record_bytes(int nl) {
  const size_t b = kModelSlot + sizeof(QHead) + (size_t)nl * kQArrays * 8;
  return (b + kRecUnit - 1) / kRecUnit * kRecUnit;
}

// What the fold kernel reports for a query it touched.
struct QPlan {
  int32_t version, done, L, pad;
  uint64_t dN[kQLevels];   // samples of the current pass, by level (0 where none)
  mlmc_result result;      // the final result once done
};

struct QView {
  QHead* h;
  double (*S)[12];
  uint64_t *n, *bad, *steps, *Ndone, *target, *dN;
};

__host__ __device__ inline QView qview(char* rec) {
  QView v;
  v.h = (QHead*)(rec + kModelSlot);
  const int nl = v.h->nl;
  char* a = rec + kModelSlot + sizeof(QHead);
  v.S = (double (*)[12])a;
  a += (size_t)nl * 12 * 8;
  uint64_t* u = (uint64_t*)a;
  v.n = u; v.bad = u + nl; v.steps = u + 2 * nl; v.Ndone = u + 3 * nl;
  v.target = u + 4 * nl; v.dN = u + 5 * nl;
  return v;
}

__device__ __forceinline__ double qsteps(const QHead* h, int l) {
  const int64_t M = (int64_t)h->M0 << l;
  return l > h->lmin ? (double)(M + M / 2) : (double)M;
}

// The driver of mlmc_estimate after a completed pass (Giles 2008, Section
// 5): after a new level's n_init samples, N_l = ceil(2 eps^-2 sqrt(V_l / C_l)
// sum_k sqrt(V_k C_k)) for every level; when nothing more is due, the bias
// test max(|Yhat_{L-1}| / 2, |Yhat_L|) < eps / sqrt(2) ends the estimate or
// adds a level.  Sets the samples of the next pass and their targets.
__device__ void qdriver(QView& v) {
  QHead* h = v.h;
  const int lmin = h->lmin;
  bool more = false;
  for (int i = 0; i < h->nl; ++i) v.dN[i] = 0;   // the completed pass's plan is spent
  if (h->pass == 0) {
    double V[kQLevels], C[kQLevels], total = 0.0;
    for (int l = lmin; l <= h->L; ++l) {
      const int i = l - lmin;
      const double n = (double)v.n[i];
      const double m1 = v.S[i][0], m2 = v.S[i][1];
      V[i] = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      if (V[i] < 0.0) V[i] = 0.0;
      C[i] = qsteps(h, l);
      total += sqrt(V[i] * C[i]);
    }
    for (int l = lmin; l <= h->L; ++l) {
      const int i = l - lmin;
      const double Nopt = ceil(2.0 / (h->eps * h->eps) * sqrt(V[i] / C[i]) * total);
      v.dN[i] = Nopt > (double)v.Ndone[i] ? (uint64_t)(Nopt - (double)v.Ndone[i]) : 0;
      more |= v.dN[i] != 0;
    }
    h->pass = 1;
  }
  if (!more) {
    bool conv = false;
    if (h->L >= lmin + 2) {
      const int i = h->L - lmin;
      const double yL = fabs(v.S[i][0] / (double)v.n[i]);
      const double yL1 = fabs(v.S[i - 1][0] / (double)v.n[i - 1]);
      conv = fmax(yL1 / 2.0, yL) < h->eps / sqrt(2.0);
    }
    if (conv || h->L >= h->Lmax) {
      h->converged = conv ? 1 : 0;
      h->done = 1;
    } else {
      h->L += 1;
      v.dN[h->L - lmin] = (uint64_t)h->n_init;
      h->pass = 0;
    }
  }
  for (int i = 0; i < h->nl; ++i) v.target[i] = v.Ndone[i] + v.dN[i];
  h->version += 1;
}

__device__ void qresult(const QView& v, mlmc_result* out) {
  const QHead* h = v.h;
  // cleared in 8-byte words (one thread: a byte-wise memset is many times slower)
  static_assert(sizeof(mlmc_result) % 8 == 0, "result in 8-byte words");
  for (size_t k = 0; k < sizeof(mlmc_result) / 8; ++k) ((unsigned long long*)out)[k] = 0ull;
  out->L = h->L;
  out->converged = h->converged;
  for (int k = 0; k < 2; ++k) {
    double est = 0.0, var = 0.0;
    for (int l = h->lmin; l <= h->L; ++l) {
      const int i = l - h->lmin;
      const double n = (double)v.n[i];
      const double m1 = v.S[i][6 * k], m2 = v.S[i][6 * k + 1];
      est += m1 / n;
      const double vv = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      var += (vv > 0.0 ? vv : 0.0) / n;
    }
    out->estimate[k] = est;
    out->est_variance[k] = var;
  }
  for (int l = h->lmin; l <= h->L; ++l) {
    const int i = l - h->lmin;
    const double n = (double)v.n[i];
    out->N[l] = v.n[i];
    out->mean_y[l] = v.S[i][0] / n;
    const double vv = n > 1.0 ? (v.S[i][1] - v.S[i][0] * v.S[i][0] / n) / (n - 1.0) : 0.0;
    out->V[l] = vv > 0.0 ? vv : 0.0;
    out->total_path_steps += v.steps[i];
    out->n_nonfinite += v.bad[i];
  }
}

// One thread per query of a launch (its requests are consecutive in the
// table, in chunk order): fold the chunks' sums into the query's record in
// that order, run the driver once the pass is complete, report the plan.
__global__ void k_serve_fold(char* __restrict__ pool, const PlanReq* __restrict__ reqs,
                             const mlmc_level_result* __restrict__ res,
                             const uint32_t* __restrict__ group_start, int n_groups,
                             QPlan* __restrict__ out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const uint32_t k0 = group_start[g], k1 = group_start[g + 1];
  QView v = qview(pool + (size_t)reqs[k0].slot * kRecUnit);
  QHead* h = v.h;
  for (uint32_t k = k0; k < k1; ++k) {
    const int i = reqs[k].level - h->lmin;
    for (int a = 0; a < 2; ++a)
      for (int j = 0; j < 6; ++j) v.S[i][6 * a + j] += res[k].sum[a][j];
    v.n[i] += res[k].n;
    v.bad[i] += res[k].n_nonfinite;
    v.steps[i] += res[k].path_steps;
    v.Ndone[i] += reqs[k].count;
  }
  bool complete = true;
  for (int i = 0; i < h->nl; ++i) complete &= v.Ndone[i] == v.target[i];
  if (complete && !h->done) qdriver(v);
  QPlan& o = out[g];
  o.version = h->version;
  o.done = h->done;
  o.L = h->L;
  o.pad = 0;
  for (int l = 0; l < kQLevels; ++l) {
    const int i = l - h->lmin;
    o.dN[l] = (i >= 0 && i < h->nl) ? v.dN[i] : 0;
  }
  if (h->done) qresult(v, &o.result);
}

struct Query {
  uint64_t id = 0;
  mlmc_params p;
  double eps = 0;
  HostModel hm;
  size_t off = 0, bytes = 0;  // record in the pool
  int nl = 0;
  int state = 0;  // 0 queued, 1 active, 2 done
  int L = 0, version = 0;
  // samples of the current pass still to issue, and the next sample to issue
  uint64_t dN[kQLevels] = {0}, Nnext[kQLevels] = {0};
  int inflight = 0;  // chunks issued and not yet folded
  int skipped = 0;   // launches in a row this query waited with work pending
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

// Paths of one chunk of level l: kChunkSteps worth, at least one full item.
static uint64_t chunk_paths(const Query& q, int l, uint64_t min_item) {
  const double c = std::floor(kChunkSteps / (double)q_steps(q, l));
  return c < (double)min_item ? min_item : (uint64_t)c;
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
  if (item_paths > 0x7FFFFFFFull) item_paths = 0x7FFFFFFFull - 0x7FFFFFFFull % min_item;
  PlanReq r;
  r.level = l;
  r.coupled = l > q.p.level_min;
  r.single = 0;
  r.M = (int64_t)q.p.M0 << l;
  r.h = q.p.T / (double)r.M;
  r.first = first;
  r.count = count;
  r.path_steps = count * spp;
  r.item_paths = (uint32_t)item_paths;
  r.n_items = (uint32_t)((count + item_paths - 1) / item_paths);
  r.item_base = 0;
  r.slot = (uint32_t)(q.off / kRecUnit);
  return r;
}

}  // namespace mlmc

using namespace mlmc;

// One launch in flight: its own stream, request table, partials, results,
// the per-query groups of its table and the plans the fold reports.
// Launches are folded, and their plans read, in issue order.
struct Flight {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;     // kernel and reduction finished (flight stream)
  cudaEvent_t folded = nullptr;   // folded and plans copied back (fold stream)
  unsigned int* d_counter = nullptr;
  PlanReq* d_reqs = nullptr;
  mlmc_level_result* d_results = nullptr;
  Partial* d_partials = nullptr;
  uint32_t* d_groups = nullptr;
  QPlan* d_plans = nullptr;
  PlanReq* h_reqs = nullptr;      // pinned
  uint32_t* h_groups = nullptr;   // pinned
  QPlan* h_plans = nullptr;       // pinned
  std::vector<uint64_t> group_query;  // the query of each group
  std::vector<int> group_chunks;      // its chunks in this launch
  int n_req = 0, n_groups = 0;
};

struct mlmc_server_s {
  int integ = 0, prec = 0, max_active = 0, grid = 0;
  uint64_t seed = 0;
  char* d_pool = nullptr;                    // query records, in the caller's workspace
  size_t pool_bytes = 0, pool_used = 0;
  std::vector<std::pair<size_t, size_t>> free_list;  // (offset, bytes), by offset
  char* h_stage = nullptr;                   // pinned staging of new records
  size_t stage_bytes = 0, stage_used = 0;
  cudaStream_t up_st = nullptr;              // record uploads
  cudaEvent_t up_ev = nullptr;               // after the latest upload
  cudaStream_t fold_st = nullptr;            // folds, in issue order
  Flight fl[kInFlight];
  std::deque<int> busy;                      // flights in flight, oldest first
  std::vector<int> idle;
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Query> q;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;              // admission order
  std::vector<std::pair<uint64_t, size_t>> to_upload;  // admitted: (query, staging offset)
  int failed = MLMC_OK;                      // first CUDA error: the server stops
  // statistics
  uint64_t ticks = 0, path_steps = 0, completed = 0;
  double busy_s = 0.0;
};

static size_t align_up(size_t b) { return (b + kRecUnit - 1) / kRecUnit * kRecUnit; }

static size_t flight_bytes() {
  return 256 + align_up((size_t)kMaxTableReq * sizeof(PlanReq)) +
         align_up((size_t)kMaxTableReq * sizeof(mlmc_level_result)) +
         (size_t)kMaxItems * sizeof(Partial) + align_up((size_t)(kMaxTableReq + 1) * 4) +
         align_up((size_t)kMaxTableReq * sizeof(QPlan));
}

static size_t fixed_bytes() { return (size_t)kInFlight * flight_bytes(); }

static int query_levels(const mlmc_params* p) { return p->L_max - p->level_min + 1; }

static void server_free(mlmc_server_s* s) {
  for (Flight& f : s->fl) {
    if (f.st) cudaStreamSynchronize(f.st);
  }
  if (s->fold_st) cudaStreamSynchronize(s->fold_st);
  for (Flight& f : s->fl) {
    if (f.done) cudaEventDestroy(f.done);
    if (f.folded) cudaEventDestroy(f.folded);
    if (f.st) cudaStreamDestroy(f.st);
    if (f.h_reqs) cudaFreeHost(f.h_reqs);
    if (f.h_groups) cudaFreeHost(f.h_groups);
    if (f.h_plans) cudaFreeHost(f.h_plans);
  }
  if (s->up_st) cudaStreamSynchronize(s->up_st);
  if (s->up_ev) cudaEventDestroy(s->up_ev);
  if (s->up_st) cudaStreamDestroy(s->up_st);
  if (s->fold_st) cudaStreamDestroy(s->fold_st);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  delete s;
}

// First fit in the pool's free list; false when no block is large enough.
static bool pool_take(mlmc_server_s* s, size_t bytes, size_t* off) {
  for (size_t k = 0; k < s->free_list.size(); ++k) {
    auto& b = s->free_list[k];
    if (b.second < bytes) continue;
    *off = b.first;
    b.first += bytes;
    b.second -= bytes;
    if (b.second == 0) s->free_list.erase(s->free_list.begin() + (long)k);
    s->pool_used += bytes;
    return true;
  }
  return false;
}

// Return a block, merging it with free neighbours.
static void pool_give(mlmc_server_s* s, size_t off, size_t bytes) {
  auto& fl = s->free_list;
  auto it = std::lower_bound(fl.begin(), fl.end(), std::make_pair(off, (size_t)0));
  it = fl.insert(it, {off, bytes});
  if (it + 1 != fl.end() && it->first + it->second == (it + 1)->first) {
    it->second += (it + 1)->second;
    fl.erase(it + 1);
  }
  if (it != fl.begin() && (it - 1)->first + (it - 1)->second == it->first) {
    (it - 1)->second += it->second;
    fl.erase(it);
  }
  s->pool_used -= bytes;
}

static double pending_steps(const Query& q) {
  double w = 0.0;
  for (int l = q.p.level_min; l <= q.L; ++l) w += (double)q.dN[l] * (double)q_steps(q, l);
  return w;
}

// Retire a finished query: its record back to the pool, statistics.
static void retire(mlmc_server_s* s, Query& qq, const mlmc_result& res, int* done) {
  qq.t_done = now_s();
  qq.result = res;
  qq.result.seconds = qq.t_done - qq.t_submit;
  qq.status = res.n_nonfinite ? MLMC_ENONFINITE : (res.converged ? MLMC_OK : MLMC_ENOTCONV);
  qq.state = 2;
  pool_give(s, qq.off, qq.bytes);
  ++*done;
  ++s->completed;
}

// Take the oldest flight's plans (waiting for its fold when `wait`); false
// when there is none or its fold has not completed.  A query whose plan has
// a new version starts the pass the device planned; a done query finishes.
static int fold_oldest(mlmc_server_s* s, bool wait, bool* folded, int* done) {
  *folded = false;
  if (s->busy.empty()) return MLMC_OK;
  Flight& f = s->fl[s->busy.front()];
  if (wait) {
    int rc = cuda_status(cudaEventSynchronize(f.folded));
    if (rc) return rc;
  } else {
    const cudaError_t e = cudaEventQuery(f.folded);
    if (e == cudaErrorNotReady) return MLMC_OK;
    if (e != cudaSuccess) return MLMC_ECUDA;
  }
  for (int g = 0; g < f.n_groups; ++g) {
    Query& qq = s->q[f.group_query[g]];
    const QPlan& pl = f.h_plans[g];
    qq.inflight -= f.group_chunks[g];
    if (pl.done) {
      retire(s, qq, pl.result, done);
    } else if (pl.version != qq.version) {
      qq.version = pl.version;
      qq.L = pl.L;
      for (int l = 0; l < kQLevels; ++l) qq.dN[l] = pl.dN[l];
    }
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

// Queued queries are admitted in arrival order while a record of their size
// fits in the pool (and fewer than max_active are active); the head of the
// queue waits for memory rather than being overtaken.
static void admit(mlmc_server_s* s) {
  while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
    Query& qq = s->q[s->queue.front()];
    if (s->stage_used + qq.bytes > s->stage_bytes) break;   // staging full until the next upload
    size_t off;
    if (!pool_take(s, qq.bytes, &off)) break;
    s->queue.pop_front();
    qq.off = off;
    qq.state = 1;
    qq.t_admit = now_s();
    qq.L = qq.p.level_min;
    qq.version = 1;
    qq.dN[qq.L] = (uint64_t)qq.p.n_init;
    // the record: Model, header, per-level arrays (zero except the first pass)
    char* rec = s->h_stage + s->stage_used;
    std::memset(rec, 0, qq.bytes);
    model_image(s->prec, qq.hm, rec);
    QHead* h = (QHead*)(rec + kModelSlot);
    h->lmin = qq.p.level_min;
    h->Lmax = qq.p.L_max;
    h->nl = qq.nl;
    h->n_init = qq.p.n_init;
    h->L = qq.p.level_min;
    h->version = 1;
    h->M0 = qq.p.M0;
    h->eps = qq.eps;
    QView v = qview(rec);
    v.dN[0] = (uint64_t)qq.p.n_init;
    v.target[0] = (uint64_t)qq.p.n_init;
    s->to_upload.push_back({qq.id, s->stage_used});
    s->stage_used += qq.bytes;
    s->active.push_back(qq.id);
  }
}

// Fill an idle flight with chunks -- least pending work first (a query's
// key halves for every launch it waited), up to the path-step budget, the
// request table and the item table -- and launch it, then its fold.
// *launched is false when no query has work to issue.
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
  f.group_query.clear();
  f.group_chunks.clear();
  int n_req = 0, n_groups = 0;
  uint64_t items = 0;
  double steps = 0.0, chain_cap = 0.0;
  bool full = false;
  for (const auto& o : order) {
    Query& qq = s->q[s->active[o.second]];
    int got = 0;
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
        if (got == 0) {                      // a new group: this query's first chunk here
          f.h_groups[n_groups++] = (uint32_t)n_req;
          f.group_query.push_back(qq.id);
          f.group_chunks.push_back(0);
        }
        r.item_base = (uint32_t)items;
        items += r.n_items;
        steps += (double)r.path_steps;
        f.h_reqs[n_req++] = r;
        f.group_chunks.back() += 1;
        qq.Nnext[l] += count;
        qq.dN[l] -= count;
        qq.inflight += 1;
        s->path_steps += r.path_steps;
        ++got;
      }
    }
    qq.skipped = got ? 0 : qq.skipped + 1;
  }
  f.h_groups[n_groups] = (uint32_t)n_req;
  f.n_req = n_req;
  f.n_groups = n_groups;
  s->idle.pop_back();
  s->busy.push_back(fi);
  int rc = MLMC_OK;
  // records of newly admitted queries go up on their own stream; every
  // launch waits for the latest upload
  if (!s->to_upload.empty()) {
    for (const auto& u : s->to_upload) {
      const Query& qq = s->q[u.first];
      if (!rc) rc = cuda_status(cudaMemcpyAsync(s->d_pool + qq.off, s->h_stage + u.second,
                                                qq.bytes, cudaMemcpyHostToDevice, s->up_st));
    }
    s->to_upload.clear();
    if (!rc) rc = cuda_status(cudaEventRecord(s->up_ev, s->up_st));
    // the staging buffer is reused once these copies have read it
    if (!rc) rc = cuda_status(cudaEventSynchronize(s->up_ev));
    s->stage_used = 0;
  }
  if (!rc) rc = cuda_status(cudaStreamWaitEvent(f.st, s->up_ev, 0));
  if (!rc) rc = cuda_status(cudaMemcpyAsync(f.d_reqs, f.h_reqs, n_req * sizeof(PlanReq),
                                            cudaMemcpyHostToDevice, f.st));
  if (!rc) rc = cuda_status(cudaMemcpyAsync(f.d_groups, f.h_groups, (n_groups + 1) * 4,
                                            cudaMemcpyHostToDevice, f.st));
  if (!rc) rc = cuda_status(cudaMemsetAsync(f.d_counter, 0, sizeof(unsigned int), f.st));
  if (!rc) rc = cuda_status(launch_multilevel_table_variant(kServeVariant, s->prec, s->integ,
                                                            s->d_pool, kRecUnit, f.d_reqs, n_req,
                                                            (uint32_t)items, f.d_partials,
                                                            f.d_counter, s->grid, f.st));
  if (!rc) rc = cuda_status(launch_finalize_table(f.d_partials, f.d_reqs, n_req, f.d_results, f.st));
  if (!rc) rc = cuda_status(cudaEventRecord(f.done, f.st));
  // the fold stream takes the launches in issue order
  if (!rc) rc = cuda_status(cudaStreamWaitEvent(s->fold_st, f.done, 0));
  if (!rc) {
    k_serve_fold<<<(n_groups + 127) / 128, 128, 0, s->fold_st>>>(s->d_pool, f.d_reqs, f.d_results,
                                                                   f.d_groups, n_groups, f.d_plans);
    rc = cuda_status(cudaGetLastError());
  }
  if (!rc) rc = cuda_status(cudaMemcpyAsync(f.h_plans, f.d_plans, n_groups * sizeof(QPlan),
                                            cudaMemcpyDeviceToHost, s->fold_st));
  if (!rc) rc = cuda_status(cudaEventRecord(f.folded, s->fold_st));
  *launched = rc == MLMC_OK;
  return rc;
}

extern "C" {

size_t mlmc_server_workspace_bytes(int max_active) {
  if (max_active < 0) return 0;
  return fixed_bytes() + (size_t)max_active * record_bytes(kSizingLevels);
}

size_t mlmc_server_query_bytes(const mlmc_params* p) {
  if (!p || p->L_max < p->level_min || p->level_min < 0 || p->L_max >= MLMC_MAX_LEVELS) return 0;
  return record_bytes(query_levels(p));
}

int mlmc_server_create(int integrator, int precision, int max_active, uint64_t seed,
                       void* workspace, size_t ws_bytes, void* stream, mlmc_server* out) {
  if (!out) return MLMC_EINVAL;
  *out = nullptr;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB) return MLMC_EINVAL;
  if (precision != MLMC_FP32 && precision != MLMC_FP64) return MLMC_EINVAL;
  if (max_active < 1 || max_active > 65536) return MLMC_EINVAL;
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < fixed_bytes() + record_bytes(3))
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
  s->d_pool = b + fixed_bytes();
  s->pool_bytes = (ws_bytes - fixed_bytes()) / kRecUnit * kRecUnit;
  s->free_list.push_back({0, s->pool_bytes});
  s->stage_bytes = std::min(s->pool_bytes, (size_t)4 << 20);
  bool ok = cudaHostAlloc((void**)&s->h_stage, s->stage_bytes, cudaHostAllocDefault) ==
                cudaSuccess &&
            cudaStreamCreateWithFlags(&s->up_st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->fold_st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&s->up_ev, cudaEventDisableTiming) == cudaSuccess;
  // work the caller queued on its stream (e.g. clearing the workspace)
  // comes before anything the server launches
  cudaEvent_t start = nullptr;
  ok = ok && cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventRecord(start, (cudaStream_t)stream) == cudaSuccess &&
       cudaStreamWaitEvent(s->up_st, start, 0) == cudaSuccess &&
       cudaStreamWaitEvent(s->fold_st, start, 0) == cudaSuccess &&
       cudaEventRecord(s->up_ev, s->up_st) == cudaSuccess;
  for (int k = 0; k < kInFlight && ok; ++k) {
    Flight& f = s->fl[k];
    f.d_counter = (unsigned int*)b;
    b += 256;
    f.d_reqs = (PlanReq*)b;
    b += align_up((size_t)kMaxTableReq * sizeof(PlanReq));
    f.d_results = (mlmc_level_result*)b;
    b += align_up((size_t)kMaxTableReq * sizeof(mlmc_level_result));
    f.d_partials = (Partial*)b;
    b += (size_t)kMaxItems * sizeof(Partial);
    f.d_groups = (uint32_t*)b;
    b += align_up((size_t)(kMaxTableReq + 1) * 4);
    f.d_plans = (QPlan*)b;
    b += align_up((size_t)kMaxTableReq * sizeof(QPlan));
    ok = cudaStreamCreateWithFlags(&f.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&f.folded, cudaEventDisableTiming) == cudaSuccess &&
         cudaHostAlloc((void**)&f.h_reqs, kMaxTableReq * sizeof(PlanReq), cudaHostAllocDefault) ==
             cudaSuccess &&
         cudaHostAlloc((void**)&f.h_groups, (kMaxTableReq + 1) * 4, cudaHostAllocDefault) ==
             cudaSuccess &&
         cudaHostAlloc((void**)&f.h_plans, kMaxTableReq * sizeof(QPlan), cudaHostAllocDefault) ==
             cudaSuccess &&
         cudaStreamWaitEvent(f.st, start, 0) == cudaSuccess;
    s->idle.push_back(kInFlight - 1 - k);
  }
  if (start) cudaEventDestroy(start);
  if (!ok) {
    server_free(s);
    return MLMC_ECUDA;
  }
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
  qq.nl = query_levels(p);
  qq.bytes = record_bytes(qq.nl);
  if (qq.bytes > s->pool_bytes || qq.bytes > s->stage_bytes) return MLMC_EWORKSPACE;
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

// One scheduling step: take the folded launches, admit, and put one more
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

int mlmc_server_pool(mlmc_server s, uint64_t out[2]) {
  if (!s || !out) return MLMC_EINVAL;
  out[0] = s->pool_used;
  out[1] = s->pool_bytes;
  return MLMC_OK;
}

int mlmc_server_destroy(mlmc_server s) {
  if (!s) return MLMC_OK;
  server_free(s);
  return MLMC_OK;
}

}  // extern "C"
