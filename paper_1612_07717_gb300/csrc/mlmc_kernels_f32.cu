// mlmc_kernels_f32.cu -- float-precision instantiation of the path kernels.
#include <cstring>

#include "mlmc_kernels.cuh"

namespace mlmc {
namespace prec_f32 {
cudaError_t level_sums(int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N,
                       uint64_t offset, Partial* partials, int grid, cudaStream_t st) {
  return level_sums_impl<float>(integ, hm, lv, N, offset, partials, grid, st);
}
cudaError_t multilevel(int integ, const HostModel& hm, const ReqPlan* plan, int n_req,
                       uint32_t n_items, Partial* partials, unsigned int* counter, int grid,
                       cudaStream_t st) {
  return multilevel_impl<float>(integ, hm, plan, n_req, n_items, partials, counter, grid, st);
}
cudaError_t multilevel_dev(int integ, const HostModel& hm, const DevPlan* plan, Partial* partials,
                           unsigned int* counter, int grid, cudaStream_t st) {
  return multilevel_dev_impl<float>(integ, hm, plan, partials, counter, grid, st);
}
cudaError_t multilevel_table(int integ, const void* models, const PlanReq* reqs, int n_req,
                             uint32_t n_items, Partial* partials, unsigned int* counter, int grid,
                             cudaStream_t st) {
  return multilevel_table_impl<float>(integ, models, reqs, n_req, n_items, partials, counter, grid, st);
}
size_t model_size() { return sizeof(Model<float>); }
void model_image(const HostModel& hm, void* out) {
  const Model<float> m = make_model<float>(hm);
  memcpy(out, &m, sizeof(m));
}
cudaError_t paths(int integ, const HostModel& hm, const LevelSpec& lv, uint64_t N, uint64_t offset,
                  void* states, int32_t* flags, void* tf, void* tc, bool trace, cudaStream_t st) {
  return paths_impl<float>(integ, hm, lv, N, offset, states, flags, tf, tc, trace, st);
}
int occupancy(int integ, bool multilevel) { return blocks_per_sm_impl<float>(integ, multilevel); }
}  // namespace prec_f32
}  // namespace mlmc
