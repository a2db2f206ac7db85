// mlmc_adaptive.cu -- kernels and launchers of the adaptive, non-nested
// timesteps (Section 7.2): coupled-level sums, the persistent multi-level
// kernel and per-pair outputs, for FP32 and FP64 paths.  They reuse the
// accumulators, reductions and planning of the uniform kernels; each adds
// the integrator steps it took to its partial sums.
#define MLMC_KNS k_adapt
#include "mlmc_kernels.cuh"
#include "mlmc_adaptive.cuh"

namespace mlmc {
namespace k_adapt {

// The thread's pairs first + k, k = begin, begin + stride, ... < end, run
// back to back: a finished pair is summed and the next one started at the
// following round.  Every thread of the warp calls this (the loop condition
// is a warp vote).
template <int INTEG, typename R, bool COUPLED>
__device__ __forceinline__ void adapt_lane(const Model<R>& m, const Level<R>& lv, uint64_t first,
                                           uint64_t begin, uint64_t end, uint64_t stride,
                                           Acc& acc) {
  uint64_t k = begin;
  bool active = k < end;
  APair<R> P;
  if (active) apair_init<R, COUPLED>(m, lv, first + k, P);
  while (__any_sync(0xFFFFFFFFu, active)) {
    if (active) {
      apair_round<INTEG, R, COUPLED>(m, P);
      if (apair_done(P)) {
        apair_finish<R, COUPLED>(P);
        acc_add<R, COUPLED>(acc, m, P.f.z, P.c.z, P.bad);
        acc.steps += P.nf + P.nc;
        k += stride;
        active = k < end;
        if (active) apair_init<R, COUPLED>(m, lv, first + k, P);
      }
    }
  }
}

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_adapt_sums(const __grid_constant__ SumsArgs<R> a) {
  Acc acc;
  acc_zero(acc, a.m.qoi1_mode != 0);
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  adapt_lane<INTEG, R, COUPLED>(a.m, a.lv, a.offset,
                                (uint64_t)blockIdx.x * kBlock + threadIdx.x, a.N, stride, acc);
  block_reduce_store(acc, COUPLED, a.m.qoi1_mode != 0, a.partials + blockIdx.x);
}

// Persistent multi-level kernel: the work-item loop of k_multilevel.
template <int INTEG, typename R>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 2 : 1) k_adapt_multilevel(const __grid_constant__ MultiArgs<R> a) {
  __shared__ unsigned int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    int r = 0;
    while (r + 1 < a.n_req && it >= a.req[r + 1].item_base) ++r;
    const ReqDev<R>& rq = a.req[r];
    const uint64_t start = (uint64_t)(it - rq.item_base) * rq.item_paths;
    const uint64_t left = rq.count - start;
    const uint32_t count = (uint32_t)(left < rq.item_paths ? left : rq.item_paths);
    const Level<R> lv = rq.lv;
    Acc acc;
    acc_zero(acc, a.m.qoi1_mode != 0);
    if (lv.coupled)
      adapt_lane<INTEG, R, true>(a.m, lv, rq.first + start, threadIdx.x, count, kBlock, acc);
    else
      adapt_lane<INTEG, R, false>(a.m, lv, rq.first + start, threadIdx.x, count, kBlock, acc);
    block_reduce_store(acc, lv.coupled != 0, a.m.qoi1_mode != 0, a.partials + it);
  }
}

template <typename R>
struct AdaptPathsArgs {
  Model<R> m;
  Level<R> lv;
  uint64_t N, offset;
  R* states;        // N x 4: z_f, w_f, z_c, w_c
  int32_t* flags;   // N
  int64_t* steps;   // N x 2 or null
};

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_adapt_paths(const __grid_constant__ AdaptPathsArgs<R> a) {
  const uint64_t j = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (j >= a.N) return;
  APair<R> P;
  run_pair_adapt<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, P);
  R* o = a.states + 4 * j;
  o[0] = P.f.z; o[1] = P.f.w;
  o[2] = COUPLED ? P.c.z : R(0);
  o[3] = COUPLED ? P.c.w : R(0);
  a.flags[j] = P.bad ? 1 : 0;
  if (a.steps) {
    a.steps[2 * j] = P.nf;
    a.steps[2 * j + 1] = P.nc;
  }
}

template <typename R>
cudaError_t sums(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N, uint64_t offset,
                 Partial* partials, int grid, cudaStream_t st) {
  SumsArgs<R> a;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.partials = partials;
  if (integ == kSE) {
    if (ls.coupled) k_adapt_sums<kSE, R, true><<<grid, kBlock, 0, st>>>(a);
    else k_adapt_sums<kSE, R, false><<<grid, kBlock, 0, st>>>(a);
  } else if (integ == kGL) {
    if (ls.coupled) k_adapt_sums<kGL, R, true><<<grid, kBlock, 0, st>>>(a);
    else k_adapt_sums<kGL, R, false><<<grid, kBlock, 0, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t multilevel(int integ, const HostModel& hm, const ReqPlan* plan, int n_req,
                       uint32_t n_items, Partial* partials, unsigned int* counter, int grid,
                       cudaStream_t st) {
  MultiArgs<R> a;
  a.m = make_model<R>(hm);
  for (int r = 0; r < n_req; ++r) {
    a.req[r].lv = make_level<R>(plan[r].lv);
    a.req[r].first = plan[r].first;
    a.req[r].count = plan[r].count;
    a.req[r].item_paths = plan[r].item_paths;
    a.req[r].n_items = plan[r].n_items;
    a.req[r].item_base = plan[r].item_base;
    a.req[r].pad = 0;
  }
  a.n_req = n_req;
  a.n_items = n_items;
  a.partials = partials;
  a.counter = counter;
  if (integ == kSE) k_adapt_multilevel<kSE, R><<<grid, kBlock, 0, st>>>(a);
  else if (integ == kGL) k_adapt_multilevel<kGL, R><<<grid, kBlock, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename R>
cudaError_t paths(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                  uint64_t offset, void* states, int32_t* flags, int64_t* steps,
                  cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  AdaptPathsArgs<R> a;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.states = (R*)states;
  a.flags = flags;
  a.steps = steps;
  const dim3 g((unsigned)((N + kBlock - 1) / kBlock));
  if (integ == kSE) {
    if (ls.coupled) k_adapt_paths<kSE, R, true><<<g, kBlock, 0, st>>>(a);
    else k_adapt_paths<kSE, R, false><<<g, kBlock, 0, st>>>(a);
  } else if (integ == kGL) {
    if (ls.coupled) k_adapt_paths<kGL, R, true><<<g, kBlock, 0, st>>>(a);
    else k_adapt_paths<kGL, R, false><<<g, kBlock, 0, st>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace k_adapt

cudaError_t launch_adapt_sums(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                              uint64_t N, uint64_t offset, Partial* partials, int grid,
                              cudaStream_t st) {
  return prec ? k_adapt::sums<double>(integ, hm, lv, N, offset, partials, grid, st)
              : k_adapt::sums<float>(integ, hm, lv, N, offset, partials, grid, st);
}

cudaError_t launch_adapt_multilevel(int prec, int integ, const HostModel& hm, const ReqPlan* plan,
                                    int n_req, uint32_t n_items, Partial* partials,
                                    unsigned int* counter, int grid, cudaStream_t st) {
  return prec ? k_adapt::multilevel<double>(integ, hm, plan, n_req, n_items, partials, counter,
                                            grid, st)
              : k_adapt::multilevel<float>(integ, hm, plan, n_req, n_items, partials, counter,
                                           grid, st);
}

cudaError_t launch_adapt_paths(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                               uint64_t N, uint64_t offset, void* d_states, int32_t* d_flags,
                               int64_t* d_steps, cudaStream_t st) {
  return prec ? k_adapt::paths<double>(integ, hm, lv, N, offset, d_states, d_flags, d_steps, st)
              : k_adapt::paths<float>(integ, hm, lv, N, offset, d_states, d_flags, d_steps, st);
}

}  // namespace mlmc
