// mlmc_adaptive.cu -- kernels and launchers of the adaptive, non-nested
// timesteps (Section 7.2): coupled-level sums, the persistent multi-level
// kernel and per-pair outputs, for FP32 and FP64 paths.  They reuse the
// accumulators, reductions and planning of the uniform kernels; each adds
// the integrator steps it took to its partial sums.
//
// Pairs take very different numbers of steps, so a block hands its pairs to
// its threads dynamically: a chunk of pairs is claimed one at a time from a
// shared counter, each finished pair's end state is parked in shared memory
// at the pair's own slot, and once the chunk is done the threads add the
// slots in a fixed order (thread t: slots t, t + 256, ...).  The sums are
// therefore independent of which thread ran which pair.
#define MLMC_KNS k_adapt
#include "mlmc_kernels.cuh"
#include "mlmc_adaptive.cuh"

namespace mlmc {
namespace k_adapt {

// Pairs per chunk and the shared memory that parks their end states:
// z_f, z_c (path precision) and the steps with the diverged mark in bit 31.
template <typename R>
struct ChunkOf {
  static constexpr uint32_t kPairs = sizeof(R) == 4 ? 4096u : 2048u;
  static constexpr size_t kBytes = (size_t)kPairs * (2 * sizeof(R) + sizeof(uint32_t));
};

// Pairs [first, first + count) of one level, run by the whole block.  Every
// thread of the block calls this (it synchronises the block).
template <int INTEG, typename R, bool COUPLED>
__device__ __forceinline__ void adapt_block(const Model<R>& m, const Level<R>& lv, uint64_t first,
                                            uint64_t count, Acc& acc) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  R* s_zf = (R*)s_dyn;
  R* s_zc = s_zf + ChunkOf<R>::kPairs;
  uint32_t* s_info = (uint32_t*)(s_zc + ChunkOf<R>::kPairs);
  __shared__ unsigned int s_next;
  for (uint64_t base = 0; base < count; base += ChunkOf<R>::kPairs) {
    const uint32_t n = (uint32_t)(count - base < ChunkOf<R>::kPairs ? count - base
                                                                    : ChunkOf<R>::kPairs);
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    uint32_t k = atomicAdd(&s_next, 1u);
    bool active = k < n;
    APair<R> P;
    if (active) apair_init<R, COUPLED>(m, lv, first + base + k, P);
    // a finished pair is parked and the next one started at the next round;
    // the loop condition is a warp vote, so every lane of the warp runs it
    while (__any_sync(0xFFFFFFFFu, active)) {
      if (active) {
        apair_round<INTEG, R, COUPLED>(m, P);
        if (apair_done(P)) {
          apair_finish<R, COUPLED>(P);
          s_zf[k] = apair_zf(P);
          s_zc[k] = apair_zc(P);
          s_info[k] = (P.nf + P.nc) | (P.bad ? 0x80000000u : 0u);
          k = atomicAdd(&s_next, 1u);
          active = k < n;
          if (active) apair_init<R, COUPLED>(m, lv, first + base + k, P);
        }
      }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBlock) {
      const uint32_t info = s_info[j];
      acc_add<R, COUPLED>(acc, m, s_zf[j], s_zc[j], (info >> 31) != 0);
      acc.steps += info & 0x7FFFFFFFu;
    }
    __syncthreads();
  }
}

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_adapt_sums(const __grid_constant__ SumsArgs<R> a) {
  Acc acc;
  acc_zero(acc, a.m.qoi1_mode != 0);
  // block b takes the contiguous pairs [b per, (b + 1) per)
  const uint64_t per = (a.N + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * per;
  const uint64_t hi = lo + per < a.N ? lo + per : a.N;
  adapt_block<INTEG, R, COUPLED>(a.m, a.lv, a.offset + lo, hi > lo ? hi - lo : 0, acc);
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
    if (lv.coupled) adapt_block<INTEG, R, true>(a.m, lv, rq.first + start, count, acc);
    else adapt_block<INTEG, R, false>(a.m, lv, rq.first + start, count, acc);
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
  o[0] = apair_zf(P); o[1] = apair_wf(P);
  o[2] = COUPLED ? apair_zc(P) : R(0);
  o[3] = COUPLED ? apair_wc(P) : R(0);
  a.flags[j] = P.bad ? 1 : 0;
  if (a.steps) {
    a.steps[2 * j] = P.nf;
    a.steps[2 * j + 1] = P.nc;
  }
}

// Launch with `smem` bytes of dynamic shared memory (above the default 48 KB
// limit when the chunk needs it).
template <typename K, typename Args>
void launch_with_smem(K kernel, int grid, size_t smem, cudaStream_t st, const Args& a) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kernel<<<grid, kBlock, smem, st>>>(a);
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
  const size_t smem = ChunkOf<R>::kBytes;
  if (integ == kSE) {
    if (ls.coupled) launch_with_smem(k_adapt_sums<kSE, R, true>, grid, smem, st, a);
    else launch_with_smem(k_adapt_sums<kSE, R, false>, grid, smem, st, a);
  } else if (integ == kGL) {
    if (ls.coupled) launch_with_smem(k_adapt_sums<kGL, R, true>, grid, smem, st, a);
    else launch_with_smem(k_adapt_sums<kGL, R, false>, grid, smem, st, a);
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
    a.req[r].single = 0;
  }
  a.n_req = n_req;
  a.n_items = n_items;
  a.partials = partials;
  a.counter = counter;
  const size_t smem = ChunkOf<R>::kBytes;
  if (integ == kSE) launch_with_smem(k_adapt_multilevel<kSE, R>, grid, smem, st, a);
  else if (integ == kGL) launch_with_smem(k_adapt_multilevel<kGL, R>, grid, smem, st, a);
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

// Resident blocks per SM of the adaptive level-sums kernel (coupled form)
// with its chunk's dynamic shared memory (the attribute is raised first, as
// at launch).
template <typename R>
int sums_blocks_per_sm(int integ) {
  const size_t smem = ChunkOf<R>::kBytes;
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (integ == kSE) {
    cudaFuncSetAttribute(k_adapt_sums<kSE, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adapt_sums<kSE, R, true>, kBlock,
                                                      smem);
  } else if (integ == kGL) {
    cudaFuncSetAttribute(k_adapt_sums<kGL, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adapt_sums<kGL, R, true>, kBlock,
                                                      smem);
  }
  if (e != cudaSuccess || nb < 1) nb = 1;
  if (nb > kMaxBlocksPerSM) nb = kMaxBlocksPerSM;
  return nb;
}

// Resident blocks per SM of the adaptive multi-level kernel with its chunk's
// dynamic shared memory (the attribute is raised first, as at launch).
template <typename R>
int multi_blocks_per_sm(int integ) {
  const size_t smem = ChunkOf<R>::kBytes;
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (integ == kSE) {
    cudaFuncSetAttribute(k_adapt_multilevel<kSE, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adapt_multilevel<kSE, R>, kBlock,
                                                      smem);
  } else if (integ == kGL) {
    cudaFuncSetAttribute(k_adapt_multilevel<kGL, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adapt_multilevel<kGL, R>, kBlock,
                                                      smem);
  }
  if (e != cudaSuccess || nb < 1) nb = 1;
  if (nb > kMaxBlocksPerSM) nb = kMaxBlocksPerSM;
  return nb;
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

int adapt_sums_blocks_per_sm(int prec, int integ) {
  return prec ? k_adapt::sums_blocks_per_sm<double>(integ)
              : k_adapt::sums_blocks_per_sm<float>(integ);
}

int adapt_multi_blocks_per_sm(int prec, int integ) {
  return prec ? k_adapt::multi_blocks_per_sm<double>(integ)
              : k_adapt::multi_blocks_per_sm<float>(integ);
}

cudaError_t launch_adapt_paths(int prec, int integ, const HostModel& hm, const LevelSpec& lv,
                               uint64_t N, uint64_t offset, void* d_states, int32_t* d_flags,
                               int64_t* d_steps, cudaStream_t st) {
  return prec ? k_adapt::paths<double>(integ, hm, lv, N, offset, d_states, d_flags, d_steps, st)
              : k_adapt::paths<float>(integ, hm, lv, N, offset, d_states, d_flags, d_steps, st);
}

}  // namespace mlmc
