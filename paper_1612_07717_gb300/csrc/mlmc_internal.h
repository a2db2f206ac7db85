// mlmc_internal.h -- host-side interface between the C ABI (mlmc_api.cu) and
// the kernel translation units (one per path precision).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mlmc.h"

namespace mlmc {

constexpr int kBlock = 256;          // threads per block of every path kernel
constexpr int kMaxReq = 32;          // requests in one multi-level launch
constexpr int kMaxItems = 32768;     // work items in one multi-level launch
constexpr int kMaxPdfBins = 32;      // bins of the binned density
constexpr int kMaxBlocksPerSM = 8;   // 2048 threads / kBlock

// Partial sums of one thread block (or one work item), 128 bytes: for each
// QoI sum Y, Y^2, P_f, P_f^2, P_c, P_c^2 (the indicator's sums are integer
// counts held exactly in doubles), the finite pairs, the diverged pairs and
// the integrator steps counted on the device (adaptive timesteps; 0 when
// the step count is fixed and known on the host).
struct Partial {
  double s0[6], s1[6];
  unsigned long long n, bad, steps, pad;
};
static_assert(sizeof(Partial) == 128, "Partial layout");
static_assert(sizeof(mlmc_level_result) == 128, "mlmc_level_result layout");

// Scenario in double precision, derived once from mlmc_params.
constexpr int kMaxSmoothR = 10;
struct HostModel {
  double H, eps, A, inv_ktau, cfu, hD, hDs, qthr, z0, w0, T;
  int32_t w0_mode, coupling, drift_outside, M0, level_min;
  uint32_t stream_id;
  uint32_t rk0[10], rk1[10];
  int32_t qoi1_mode, smooth_r;        // smoothed interval QoI (Section 5.1)
  double qa, qb, delta;
  double pc[kMaxSmoothR + 2];         // p_r(s) = sum_k pc[k] s^k
  int32_t adapt;                      // adaptive timesteps (Section 7.2)
  double z_adapt, lam_a;              // X_adapt and lambda(X_adapt)
};
// Adaptive timesteps count time in units of h_l / 1024 of the level: T is
// 1024 M_l units, and a pair's steps (at most 1536 M_l) must fit 31 bits.
constexpr int64_t kAdaptMaxM = (int64_t)1 << 20;
// Coefficients of the smoothing polynomial p_r (Section 5.1); 0 or -1.
int smooth_coefficients(int r, double* c);

struct LevelSpec {
  int level;
  int64_t M;
  double h;
  bool coupled;
};

// One request of a multi-level launch after planning on the host.
// A packed (two pairs per thread) launch runs a request one pair per thread
// when one of its pairs alone is at least this share of a thread's average
// work, total path-steps / (grid * kBlock): such pairs set the launch's
// length, and one pair per thread issues about two thirds of a packed warp's
// instructions per step.
constexpr double kSingleShare = 0.25;

struct ReqPlan {
  LevelSpec lv;
  uint64_t first, count;
  uint32_t item_paths, n_items, item_base;
  uint32_t single;       // packed kernels: one pair per thread for this request's items
  uint64_t path_steps;
};

// A request of a device-planned multi-level launch (the graph-driven
// estimator plans on the device), precision independent, 64 bytes.
struct PlanReq {
  int32_t level;
  uint16_t coupled, single;   // single: packed kernels run the items one pair per thread
  int64_t M;
  double h;
  uint64_t first, count, path_steps;
  uint32_t item_paths, n_items, item_base, slot;  // slot: query of a multi-query batch
};
struct DevPlan {
  int32_t n_req;
  uint32_t n_items;
  uint32_t pad[14];
  PlanReq req[kMaxReq];
};
static_assert(sizeof(PlanReq) == 64, "PlanReq layout");

// Kernel launchers, implemented per precision (prec: 0 float, 1 double).
cudaError_t launch_level_sums(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                              uint64_t N, uint64_t offset, Partial* partials, int grid,
                              cudaStream_t st);
cudaError_t launch_multilevel(int prec, int integ, const HostModel& hm, const ReqPlan* plan,
                              int n_req, uint32_t n_items, Partial* partials,
                              unsigned int* counter, int grid, cudaStream_t st);
cudaError_t launch_multilevel_dev(int prec, int integ, const HostModel& hm, const DevPlan* plan,
                                  Partial* partials, unsigned int* counter, int grid,
                                  cudaStream_t st);
// Multi-query batches (serving): a table of requests in device memory, each
// tagged with the slot of its query's Model; slot k's Model starts at byte
// k * stride of `models`.
cudaError_t launch_multilevel_table(int prec, int integ, const void* models, size_t stride,
                                   const PlanReq* reqs, int n_req, uint32_t n_items,
                                   Partial* partials, unsigned int* counter, int grid,
                                   cudaStream_t st);
// Binned density of one level (k bins): per block 2k + 2 doubles.
cudaError_t launch_pdf(int prec, int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N,
                       uint64_t offset, int k, double* partials, int grid, cudaStream_t st);
// Adaptive timesteps (mlmc_adaptive.cu): the same launches for hm.adapt.
// Level sums and multi-level partials count the integrator steps.
cudaError_t launch_adapt_sums(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                              uint64_t N, uint64_t offset, Partial* partials, int grid,
                              cudaStream_t st);
cudaError_t launch_adapt_multilevel(int prec, int integ, const HostModel& hm, const ReqPlan* plan,
                                    int n_req, uint32_t n_items, Partial* partials,
                                    unsigned int* counter, int grid, cudaStream_t st);
// Resident blocks per SM of the adaptive level-sums and multi-level kernels.
int adapt_sums_blocks_per_sm(int prec, int integ);
int adapt_multi_blocks_per_sm(int prec, int integ);
cudaError_t launch_adapt_paths(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                               uint64_t N, uint64_t offset, void* d_states, int32_t* d_flags,
                               int64_t* d_steps, cudaStream_t st);
// Bytes of one device Model of precision prec, and its host image.
size_t model_bytes(int prec);
void model_image(int prec, const HostModel& hm, void* out);
cudaError_t launch_paths(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                         uint64_t N, uint64_t offset, void* d_states, int32_t* d_flags,
                         cudaStream_t st);
cudaError_t launch_trace(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                         uint64_t N, uint64_t offset, void* d_tf, void* d_tc, void* d_thf,
                         void* d_thc, cudaStream_t st);
// Resident blocks per SM of the sums / multi-level kernels (occupancy query
// and tuning table), and the planner's work items per resident block.
int blocks_per_sm(int prec, int integ, bool multilevel);
int items_per_block(int prec, int integ);
// Smallest work item of the planners: one pass of the block over its path
// pairs (kBlock pairs, 2 kBlock for the two-pairs-per-thread variants).
uint64_t min_item_paths(int prec, int integ);
// The query server's kernel, whatever the tuning table holds: one path pair
// per thread at 4 blocks per SM, the finest work items (latency before
// throughput); its launcher and grid.
constexpr int kServeVariant = 4;
cudaError_t launch_multilevel_table_variant(int variant, int prec, int integ, const void* models,
                                            size_t stride, const PlanReq* reqs, int n_req,
                                            uint32_t n_items, Partial* partials,
                                            unsigned int* counter, int grid, cudaStream_t st);
int grid_for_variant(int variant, int prec, int integ);

// Device facts, workspace carving and parameter handling (mlmc_api.cu).
struct DevInfo {
  int sms = 0, cc = 0;
};
// Workspace layout: [256 B header][kMaxReq results][partial slots][graph region].
constexpr size_t kGraphRegion = 16384;  // device-side MLMC driver state (mlmc_graph.cu)
struct Workspace {
  unsigned int* counter;
  mlmc_level_result* results;
  Partial* partials;
  char* graph;
};
int device_info(DevInfo* out);
size_t workspace_needed();
int carve(void* ws, size_t bytes, Workspace* w);
int make_host_model(const mlmc_params* p, uint64_t seed, HostModel* hm);
int level_spec(const HostModel& hm, int level, LevelSpec* ls);
uint64_t steps_per_pair(const LevelSpec& ls);
int check_stable(int integ, const mlmc_params* p, const HostModel& hm, const LevelSpec& ls);
int grid_for(int prec, int integ, bool multilevel, uint64_t N);
int cuda_status(cudaError_t e);

// Precision-independent reductions (mlmc_api.cu).
cudaError_t launch_finalize(const Partial* partials, int nblocks, uint64_t path_steps,
                            mlmc_level_result* d_out, cudaStream_t st);
cudaError_t launch_finalize_dev(const Partial* partials, const DevPlan* plan,
                                mlmc_level_result* d_out, cudaStream_t st);
cudaError_t launch_finalize_table(const Partial* partials, const PlanReq* reqs, int n_req,
                                  mlmc_level_result* d_out, cudaStream_t st);
cudaError_t launch_finalize_multi(const Partial* partials, const ReqPlan* plan, int n_req,
                                  mlmc_level_result* d_out, cudaStream_t st);

}  // namespace mlmc
