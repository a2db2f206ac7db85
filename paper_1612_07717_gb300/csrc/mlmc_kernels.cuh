// mlmc_kernels.cuh -- the path kernels, instantiated once per precision by
// mlmc_kernels_f32.cu and mlmc_kernels_f64.cu.
//
//   k_level_sums  coupled-level kernel: a grid-stride loop of path pairs,
//                 per-thread FP64 accumulation (Kahan on sum Y and sum Y^2),
//                 a block reduction into one Partial per block.
//   k_multilevel  persistent multi-level kernel: blocks pull fixed-size work
//                 items of any level from an atomic counter (items ordered
//                 by per-path cost, finest level first) and write one
//                 Partial per item, so the sums do not depend on scheduling.
//   k_paths       final states per pair (validation and per-particle output)
//   k_trace       full trajectories (validation)
#pragma once
#include <type_traits>

#include "mlmc_device.cuh"
#include "mlmc_internal.h"
#include "mlmc_reduce.cuh"
#if MLMC_X2
#include "mlmc_device_x2.cuh"
#endif

// Minimum resident blocks per SM requested from the register allocator for
// the path kernels (1: no register cap).  Each translation unit that
// includes this file instantiates the kernels in its own namespace
// MLMC_KNS, so variants with different register budgets can coexist.
#ifndef MLMC_MINB
#define MLMC_MINB 1
#endif
#ifndef MLMC_KNS
#define MLMC_KNS kdefault
#endif
// MLMC_X2 = 1: the FP32 persistent multi-level kernels run two path pairs
// per thread on the packed FP32 instructions (mlmc_device_x2.cuh).
#ifndef MLMC_X2
#define MLMC_X2 0
#endif

namespace mlmc {
namespace MLMC_KNS {

// ---------------------------------------------------------------------------
// Host -> device constants
// ---------------------------------------------------------------------------
template <typename R>
Model<R> make_model(const HostModel& h) {
  Model<R> m;
  m.H = (R)h.H;
  m.twoH = (R)(2.0 * h.H);
  m.eps = (R)h.eps;
  m.Hme = (R)(h.H - h.eps);
  m.invH = (R)(1.0 / h.H);
  m.A = (R)h.A;
  m.Akt = (R)(h.A * h.inv_ktau);
  m.cfu = (R)h.cfu;
  m.hD = (R)h.hD;
  m.hDs = (R)h.hDs;
  m.hD_out = h.drift_outside ? (R)h.hD : R(0);
  m.hDs_out = h.drift_outside ? (R)h.hDs : R(0);
  m.qthr = (R)h.qthr;
  m.z0 = (R)h.z0;
  m.w0 = (R)h.w0;
  m.lim = (R)(1e3 * h.H);
  m.w0_mode = h.w0_mode;
  m.coupling = h.coupling;
  m.stream_id = h.stream_id;
  m.qoi1_mode = h.qoi1_mode;
  m.sdeg = h.smooth_r + 1;
  m.qa = (R)h.qa;
  m.qb = (R)h.qb;
  m.idelta = h.delta > 0.0 ? (R)(1.0 / h.delta) : R(0);
  for (int k = 0; k < 12; ++k) m.pc[k] = (R)h.pc[k];
  for (int r = 0; r < 10; ++r) { m.rk0[r] = h.rk0[r]; m.rk1[r] = h.rk1[r]; }
  m.za = (R)h.z_adapt;
  m.lam_a = (R)h.lam_a;
  return m;
}

template <typename R>
Level<R> make_level(const LevelSpec& s) {
  Level<R> l;
  l.h = (R)s.h;
  l.h2 = (R)(0.5 * s.h);
  l.hc = (R)(2.0 * s.h);
  l.hc2 = (R)s.h;
  l.hl2 = (R)(s.h * 1.4426950408889634074);
  l.hcl2 = (R)(2.0 * s.h * 1.4426950408889634074);
  l.M = s.M;
  l.c2 = (uint32_t)s.level << 24;
  l.coupled = s.coupled ? 1 : 0;
  return l;
}

// ---------------------------------------------------------------------------
// Per-thread accumulator and block reduction
// ---------------------------------------------------------------------------
// Per-thread sums are plain FP64 (a thread adds at most a few thousand
// terms, error below 1e-12 relative); the compensation is applied where the
// partial sums of a block and of the blocks are combined.  On the coarsest
// level P_c = 0, so only sum Y and sum Y^2 are kept (sum P_f = sum Y).
// QoI 1: the indicator is counted in integers (exact); the smoothed
// interval QoI keeps its six FP64 sums per thread in shared memory (they are
// touched once per path), so it costs no registers when unused.
struct Acc {
  double y, y2, pf, pf2, pc, pc2;
  uint32_t n, bad, nf, nc, nd;
  uint64_t steps;   // integrator steps (adaptive kernels; 0 otherwise)
};

__device__ __forceinline__ double (*q1_smem())[kBlock] {
  __shared__ double s_q1[6][kBlock];
  return s_q1;
}

__device__ __forceinline__ void kahan_add(double& s, double& c, double x) {
  const double y = x - c;
  const double t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ void acc_zero(Acc& a, bool smooth) {
  a.y = a.y2 = a.pf = a.pf2 = a.pc = a.pc2 = 0.0;
  a.n = a.bad = a.nf = a.nc = a.nd = 0;
  a.steps = 0;
  if (smooth) {
    double (*q)[kBlock] = q1_smem();
    for (int k = 0; k < 6; ++k) q[k][threadIdx.x] = 0.0;
  }
}

// QoIs at T (Section 3.3): P = z(T), and P = 1[z(T) < threshold] or the
// smoothed interval; Y = P_f - P_c is formed in FP64 (exact for two floats);
// the indicator decision is taken in the path precision.
template <typename R, bool COUPLED>
__device__ __forceinline__ void acc_add(Acc& a, const Model<R>& m, R zf, R zc, bool bad) {
  if (bad) { a.bad += 1; return; }
  const double Pf = (double)zf;
  if (COUPLED) {
    const double Pc = (double)zc;
    const double Y = Pf - Pc;
    a.y += Y;
    a.y2 = fma(Y, Y, a.y2);
    a.pf += Pf;
    a.pf2 = fma(Pf, Pf, a.pf2);
    a.pc += Pc;
    a.pc2 = fma(Pc, Pc, a.pc2);
  } else {
    a.y += Pf;
    a.y2 = fma(Pf, Pf, a.y2);
  }
  if (m.qoi1_mode) {
    const double Sf = (double)smoothed_interval(m, zf);
    const double Sc = COUPLED ? (double)smoothed_interval(m, zc) : 0.0;
    const double Y1 = Sf - Sc;
    double (*q)[kBlock] = q1_smem();
    const int t = threadIdx.x;
    q[0][t] += Y1;
    q[1][t] = fma(Y1, Y1, q[1][t]);
    q[2][t] += Sf;
    q[3][t] = fma(Sf, Sf, q[3][t]);
    q[4][t] += Sc;
    q[5][t] = fma(Sc, Sc, q[5][t]);
  } else {
    const bool If = zf < m.qthr;
    const bool Ic = COUPLED && (zc < m.qthr);
    a.nf += If; a.nc += Ic; a.nd += (If != Ic);
  }
  a.n += 1;
}

// Warp tree (fixed order, warp_tree12), then the warp results are added in
// warp order with Kahan compensation, one lane of warp 0 per sum.  FP64
// instructions hold the FP64 pipe for many cycles whatever the number of
// active lanes, so the sums go side by side in the lanes rather than one after
// another in one thread; a warp whose lanes saw no pair skips its tree (its
// sums are exact zeros).  Ends with the block synchronised.
__device__ __forceinline__ void block_reduce_store(const Acc& a, bool coupled, bool smooth,
                                                   Partial* __restrict__ out) {
  // the warp trees reuse the smoothed QoI's per-thread sums (12 KB), each
  // thread reading its own sums into v before the barrier below
  double (*s_tree)[12][16] = reinterpret_cast<double (*)[12][16]>(&q1_smem()[0][0]);
  static_assert(sizeof(double) * 6 * kBlock == sizeof(double) * (kBlock / 32) * 12 * 16, "tree buffer");
  __shared__ unsigned long long s_u[kBlock / 32][3];
  double v[12] = {a.y, a.y2, coupled ? a.pf : a.y, coupled ? a.pf2 : a.y2, a.pc, a.pc2};
  if (smooth) {
    double (*q)[kBlock] = q1_smem();
#pragma unroll
    for (int k = 0; k < 6; ++k) v[6 + k] = q[k][threadIdx.x];
  } else {
    const double nf = (double)a.nf, nc = (double)a.nc, nd = (double)a.nd;
    v[6] = nf - nc; v[7] = nd; v[8] = nf; v[9] = nf; v[10] = nc; v[11] = nc;
  }
  unsigned long long u[3] = {a.n, a.bad, a.steps};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();                       // every thread has read its smoothed sums
  if (__any_sync(0xFFFFFFFFu, a.n + a.bad != 0)) {
    warp_tree12(v, s_tree[warp], lane);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) u[k] += __shfl_down_sync(0xFFFFFFFFu, u[k], off);
    }
  } else if (lane < 12) {
    s_tree[warp][lane][0] = 0.0;
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) s_u[warp][k] = u[k];
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int k = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) kahan_add(s, c, s_tree[w][k][0]);
    (k < 6 ? out->s0 : out->s1)[k < 6 ? k : k - 6] = s - c;
  } else if (threadIdx.x < 15) {
    const int k = threadIdx.x - 12;
    unsigned long long t = 0;
    for (int w = 0; w < kBlock / 32; ++w) t += s_u[w][k];
    (k == 0 ? out->n : k == 1 ? out->bad : out->steps) = t;
  } else if (threadIdx.x == 15) {
    out->pad = 0;
  }
  __syncthreads();
}

#if MLMC_X2
// Lane of a packed pair: the exact replay where the fast pass flagged a
// multi-layer step, then the finiteness check, exactly as run_pair does.
// Returns the diverged mark; the final states are updated in place.
template <int INTEG, bool COUPLED>
__device__ __forceinline__ bool lane_final(const Model<float>& m, const Level<float>& lv,
                                           uint64_t i, float& fz, float& fw, float& cz,
                                           float& cw, bool multi) {
  bool bad = false;
  if (multi) {
    Path<float> f, c;
    run_pair_impl<INTEG, float, COUPLED, true>(m, lv, i, f, c, bad, NoTrace<float>());
    fz = f.z; fw = f.w; cz = c.z; cw = c.w;
  }
  bad |= !(isfinite(fz) && isfinite(fw));
  if (COUPLED) bad |= !(isfinite(cz) && isfinite(cw));
  return bad;
}

template <int INTEG, bool COUPLED>
__device__ __forceinline__ void finish_lane(const Model<float>& m, const Level<float>& lv,
                                            uint64_t i, float fz, float fw, float cz, float cw,
                                            bool multi, Acc& acc) {
  const bool bad = lane_final<INTEG, COUPLED>(m, lv, i, fz, fw, cz, cw, multi);
  acc_add<float, COUPLED>(acc, m, fz, cz, bad);
}

// Thread t of the block takes pairs 2t and 2t + 1 of each stride of 2 kBlock
// pairs; a lane past the item's end is computed and discarded.
template <int INTEG, bool COUPLED>
__device__ __forceinline__ void multilevel_item_x2(const Model<float>& m, const Level<float>& lv,
                                                   uint64_t first, uint32_t count, Acc& acc) {
  const StartX2 s0 = start_x2(m);
  for (uint32_t j = 2 * threadIdx.x; j < count; j += 2 * kBlock) {
    PathX2 f, c;
    bool mx, my;
    run_pair_x2_fast<INTEG, COUPLED>(m, lv, s0, first + j, f, c, mx, my);
    finish_lane<INTEG, COUPLED>(m, lv, first + j, f.z.x, f.w.x, c.z.x, c.w.x, mx, acc);
    if (j + 1 < count)
      finish_lane<INTEG, COUPLED>(m, lv, first + j + 1, f.z.y, f.w.y, c.z.y, c.w.y, my, acc);
  }
}
#endif

// ---------------------------------------------------------------------------
// Coupled-level sums
// ---------------------------------------------------------------------------
template <typename R>
struct SumsArgs {
  Model<R> m;
  Level<R> lv;
  uint64_t N, offset;
  Partial* partials;
};

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock, MLMC_MINB) k_level_sums(const __grid_constant__ SumsArgs<R> a) {
  Acc acc;
  acc_zero(acc, a.m.qoi1_mode != 0);
  if constexpr (MLMC_X2 && std::is_same<R, float>::value) {
#if MLMC_X2
    // two pairs per thread: pairs 2g and 2g + 1 of global thread g, grid-stride
    const StartX2 s0 = start_x2(a.m);
    const uint64_t stride = 2 * (uint64_t)gridDim.x * kBlock;
    for (uint64_t j = 2 * ((uint64_t)blockIdx.x * kBlock + threadIdx.x); j < a.N; j += stride) {
      PathX2 f, c;
      bool mx, my;
      run_pair_x2_fast<INTEG, COUPLED>(a.m, a.lv, s0, a.offset + j, f, c, mx, my);
      finish_lane<INTEG, COUPLED>(a.m, a.lv, a.offset + j, f.z.x, f.w.x, c.z.x, c.w.x, mx, acc);
      if (j + 1 < a.N)
        finish_lane<INTEG, COUPLED>(a.m, a.lv, a.offset + j + 1, f.z.y, f.w.y, c.z.y, c.w.y, my,
                                    acc);
    }
#endif
  } else {
    const uint64_t stride = (uint64_t)gridDim.x * kBlock;
    for (uint64_t j = (uint64_t)blockIdx.x * kBlock + threadIdx.x; j < a.N; j += stride) {
      Path<R> f, c;
      bool bad;
      run_pair<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, f, c, bad, NoTrace<R>());
      acc_add<R, COUPLED>(acc, a.m, f.z, c.z, bad);
    }
  }
  block_reduce_store(acc, COUPLED, a.m.qoi1_mode != 0, a.partials + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Persistent multi-level kernel
// ---------------------------------------------------------------------------
template <typename R>
struct ReqDev {
  Level<R> lv;
  uint64_t first, count;
  uint32_t item_paths, n_items, item_base, single;
};

template <typename R>
struct MultiArgs {
  Model<R> m;
  ReqDev<R> req[kMaxReq];
  int32_t n_req;
  uint32_t n_items;
  Partial* partials;
  unsigned int* counter;
};


// `single` (packed kernels only) runs the item one pair per thread on the
// scalar path: a warp of the launch's longest pairs then issues about two
// thirds of the instructions per step, which shortens a launch whose finest
// level outlasts the rest of the work.  Both paths give the same pairs bit for
// bit.
template <int INTEG, typename R, bool COUPLED>
__device__ __forceinline__ void multilevel_item(const Model<R>& m, const Level<R> lv,
                                                uint64_t first, uint32_t count, bool single,
                                                Acc& acc) {
  if constexpr (MLMC_X2 && std::is_same<R, float>::value) {
#if MLMC_X2
    if (!single) {
      multilevel_item_x2<INTEG, COUPLED>(m, lv, first, count, acc);
      return;
    }
#endif
  }
  {
    for (uint32_t j = threadIdx.x; j < count; j += kBlock) {
      Path<R> f, c;
      bool bad;
      run_pair<INTEG, R, COUPLED>(m, lv, first + j, f, c, bad, NoTrace<R>());
      acc_add<R, COUPLED>(acc, m, f.z, c.z, bad);
    }
  }
}

template <int INTEG, typename R>
__global__ void __launch_bounds__(kBlock, MLMC_MINB) k_multilevel(const __grid_constant__ MultiArgs<R> a) {
  __shared__ unsigned int s_item;
  // Every block does at most n_items iterations: the loop ends when the
  // shared counter passes the last item; there is no waiting on other blocks.
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= a.n_items) break;
    int r = 0;
    while (r + 1 < a.n_req && it >= a.req[r + 1].item_base) ++r;
    const ReqDev<R>& rq = a.req[r];
    const uint32_t local = it - rq.item_base;
    const uint64_t start = (uint64_t)local * rq.item_paths;
    const uint64_t left = rq.count - start;
    const uint32_t count = (uint32_t)(left < rq.item_paths ? left : rq.item_paths);
    Acc acc;
    acc_zero(acc, a.m.qoi1_mode != 0);
    const Level<R> lv = rq.lv;   // registers, not parameter-space loads per step
    if (lv.coupled)
      multilevel_item<INTEG, R, true>(a.m, lv, rq.first + start, count, rq.single != 0, acc);
    else
      multilevel_item<INTEG, R, false>(a.m, lv, rq.first + start, count, rq.single != 0, acc);
    block_reduce_store(acc, lv.coupled != 0, a.m.qoi1_mode != 0, a.partials + it);
  }
}

// The same persistent kernel with its plan in device memory (written by the
// device-side MLMC driver between launches of a captured graph).
template <int INTEG, typename R>
__global__ void __launch_bounds__(kBlock, MLMC_MINB) k_multilevel_dev(const __grid_constant__ Model<R> m,
                                                           const DevPlan* __restrict__ plan,
                                                           Partial* __restrict__ partials,
                                                           unsigned int* __restrict__ counter) {
  __shared__ unsigned int s_item;
  const int n_req = plan->n_req;
  const uint32_t n_items = plan->n_items;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const unsigned int it = s_item;
    __syncthreads();
    if (it >= n_items) break;
    int r = 0;
    while (r + 1 < n_req && it >= plan->req[r + 1].item_base) ++r;
    const PlanReq& pr = plan->req[r];
    ReqDev<R> rq;
    rq.lv.h = (R)pr.h;
    rq.lv.h2 = (R)(0.5 * pr.h);
    rq.lv.hc = (R)(2.0 * pr.h);
    rq.lv.hc2 = (R)pr.h;
    rq.lv.hl2 = (R)(pr.h * 1.4426950408889634074);
    rq.lv.hcl2 = (R)(2.0 * pr.h * 1.4426950408889634074);
    rq.lv.M = pr.M;
    rq.lv.c2 = (uint32_t)pr.level << 24;
    rq.lv.coupled = pr.coupled;
    rq.first = pr.first;
    rq.count = pr.count;
    rq.item_paths = pr.item_paths;
    rq.single = pr.single;
    const uint32_t local = it - pr.item_base;
    const uint64_t start = (uint64_t)local * pr.item_paths;
    const uint64_t left = pr.count - start;
    const uint32_t count = (uint32_t)(left < pr.item_paths ? left : pr.item_paths);
    Acc acc;
    acc_zero(acc, m.qoi1_mode != 0);
    if (pr.coupled)
      multilevel_item<INTEG, R, true>(m, rq.lv, pr.first + start, count, pr.single != 0, acc);
    else
      multilevel_item<INTEG, R, false>(m, rq.lv, pr.first + start, count, pr.single != 0, acc);
    block_reduce_store(acc, pr.coupled != 0, m.qoi1_mode != 0, partials + it);
  }
}

// Multi-query batches: the request table lives in device memory and each
// request names the slot of its query's Model.  Items of different queries
// share one launch; each request's items are reduced in item order, and the
// item split of a request does not depend on the rest of the batch, so a
// query's sums are the same alone and in any mix.
template <int INTEG, typename R>
__global__ void __launch_bounds__(kBlock, MLMC_MINB)
    k_multilevel_table(const char* __restrict__ models, size_t model_stride,
                       const PlanReq* __restrict__ reqs, int n_req, uint32_t n_items,
                       Partial* __restrict__ partials, unsigned int* __restrict__ counter) {
  __shared__ unsigned int s_item;
  __shared__ int s_req;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int it = atomicAdd(counter, 1u);
      int lo = 0, hi = n_req - 1;                    // last request with item_base <= it
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].item_base <= it) lo = mid; else hi = mid - 1;
      }
      s_item = it;
      s_req = lo;
    }
    __syncthreads();
    const unsigned int it = s_item;
    const int r = s_req;
    __syncthreads();
    if (it >= n_items) break;
    const PlanReq pr = reqs[r];
    const Model<R> m = *(const Model<R>*)(models + (size_t)pr.slot * model_stride);
    Level<R> lv;
    lv.h = (R)pr.h;
    lv.h2 = (R)(0.5 * pr.h);
    lv.hc = (R)(2.0 * pr.h);
    lv.hc2 = (R)pr.h;
    lv.hl2 = (R)(pr.h * 1.4426950408889634074);
    lv.hcl2 = (R)(2.0 * pr.h * 1.4426950408889634074);
    lv.M = pr.M;
    lv.c2 = (uint32_t)pr.level << 24;
    lv.coupled = pr.coupled;
    const uint32_t local = it - pr.item_base;
    const uint64_t start = (uint64_t)local * pr.item_paths;
    const uint64_t left = pr.count - start;
    const uint32_t count = (uint32_t)(left < pr.item_paths ? left : pr.item_paths);
    Acc acc;
    acc_zero(acc, m.qoi1_mode != 0);
    if (pr.coupled)
      multilevel_item<INTEG, R, true>(m, lv, pr.first + start, count, pr.single != 0, acc);
    else
      multilevel_item<INTEG, R, false>(m, lv, pr.first + start, count, pr.single != 0, acc);
    block_reduce_store(acc, pr.coupled != 0, m.qoi1_mode != 0, partials + it);
  }
}

// ---------------------------------------------------------------------------
// Binned density (Section 6.3, Eq. vector_QoI): k bins [i w, (i+1) w),
// w = H / k, each QoI the smoothed interval of its bin.  With edge values
// G_e = g_r((z - e w) / delta), bin i's QoI is G_{i+1} - G_i.  Per thread the
// sums of Y_i and Y_i^2 sit in dynamic shared memory ([2k][256] doubles);
// each block writes 2k + 2 doubles (the sums, then the finite and the
// diverged pair counts) to its own slot.
// ---------------------------------------------------------------------------
template <typename R>
struct PdfArgs {
  Model<R> m;
  Level<R> lv;
  uint64_t N, offset;
  int32_t k;
  R binw;
  double* partials;   // gridDim.x x (2k + 2)
};

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_level_pdf(const __grid_constant__ PdfArgs<R> a) {
  extern __shared__ double s_pdf[];   // [2k][kBlock]
  const int t = threadIdx.x;
  const int k = a.k;
  for (int c = 0; c < 2 * k; ++c) s_pdf[c * kBlock + t] = 0.0;
  double n_ok = 0.0, n_bad = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t j = (uint64_t)blockIdx.x * kBlock + t; j < a.N; j += stride) {
    Path<R> f, c;
    bool bad;
    run_pair<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, f, c, bad, NoTrace<R>());
    if (bad) { n_bad += 1.0; continue; }
    n_ok += 1.0;
    R gf0 = g_smooth(a.m, f.z * a.m.idelta);
    R gc0 = COUPLED ? g_smooth(a.m, c.z * a.m.idelta) : R(0);
    for (int i = 0; i < k; ++i) {
      const R e = (R)(i + 1) * a.binw;
      const R gf1 = g_smooth(a.m, (f.z - e) * a.m.idelta);
      const R gc1 = COUPLED ? g_smooth(a.m, (c.z - e) * a.m.idelta) : R(0);
      const double Y = ((double)gf1 - (double)gf0) - (COUPLED ? ((double)gc1 - (double)gc0) : 0.0);
      s_pdf[(2 * i) * kBlock + t] += Y;
      s_pdf[(2 * i + 1) * kBlock + t] = fma(Y, Y, s_pdf[(2 * i + 1) * kBlock + t]);
      gf0 = gf1;
      gc0 = gc1;
    }
  }
  // block reduction of each column: warp tree, then warp-ordered Kahan, one
  // thread per column (side by side: FP64 instructions are slow to issue)
  __shared__ double s_w[kBlock / 32][2 * kMaxPdfBins + 2];
  const int lane = t & 31, warp = t >> 5;
  double* out = a.partials + (size_t)blockIdx.x * (2 * k + 2);
  for (int col = 0; col < 2 * k + 2; ++col) {
    double v = col < 2 * k ? s_pdf[col * kBlock + t] : (col == 2 * k ? n_ok : n_bad);
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if (lane == 0) s_w[warp][col] = v;
  }
  __syncthreads();
  for (int col = t; col < 2 * k + 2; col += kBlock) {
    double s = 0.0, cc = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) kahan_add(s, cc, s_w[w][col]);
    out[col] = s - cc;
  }
}

template <int I, typename R, bool C>
struct PdfK {
  static void launch(dim3 g, const PdfArgs<R>& a, cudaStream_t st) {
    const size_t smem = (size_t)2 * a.k * kBlock * sizeof(double);
    cudaFuncSetAttribute(k_level_pdf<I, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_level_pdf<I, R, C><<<g, kBlock, smem, st>>>(a);
  }
};

// ---------------------------------------------------------------------------
// Per-path outputs
// ---------------------------------------------------------------------------
template <typename R>
struct PathsArgs {
  Model<R> m;
  Level<R> lv;
  uint64_t N, offset;
  R* states;        // N x 4
  int32_t* flags;   // N
  R* tf;            // trace: N x (M+1) x 3
  R* tc;            // trace: N x (M/2+1) x 3
  R* thf;           // half-step trace (BAOAB): N x M x 3
  R* thc;           // half-step trace (BAOAB): N x M/2 x 3
};

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_paths(const __grid_constant__ PathsArgs<R> a) {
  const uint64_t j = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (j >= a.N) return;
  Path<R> f, c;
  bool bad;
  run_pair<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, f, c, bad, NoTrace<R>());
  R* o = a.states + 4 * j;
  o[0] = f.z; o[1] = f.w;
  o[2] = COUPLED ? c.z : R(0);
  o[3] = COUPLED ? c.w : R(0);
  a.flags[j] = bad ? 1 : 0;
}

// Final states per pair through the path code of this translation unit's
// tuning variant (its register budget; two pairs per thread on the packed
// instructions in the MLMC_X2 units, thread g taking pairs 2g and 2g + 1 as
// the level-sums kernel does), so the pairs the production kernels reduce
// can be compared one by one.
template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock, MLMC_MINB) k_paths_v(const __grid_constant__ PathsArgs<R> a) {
  if constexpr (MLMC_X2 && std::is_same<R, float>::value) {
#if MLMC_X2
    const uint64_t j = 2 * ((uint64_t)blockIdx.x * kBlock + threadIdx.x);
    if (j >= a.N) return;
    const StartX2 s0 = start_x2(a.m);
    PathX2 f, c;
    bool mx, my;
    run_pair_x2_fast<INTEG, COUPLED>(a.m, a.lv, s0, a.offset + j, f, c, mx, my);
    float fz = f.z.x, fw = f.w.x, cz = c.z.x, cw = c.w.x;
    bool bad = lane_final<INTEG, COUPLED>(a.m, a.lv, a.offset + j, fz, fw, cz, cw, mx);
    R* o = a.states + 4 * j;
    o[0] = fz; o[1] = fw;
    o[2] = COUPLED ? cz : 0.0f;
    o[3] = COUPLED ? cw : 0.0f;
    a.flags[j] = bad ? 1 : 0;
    if (j + 1 < a.N) {                        // the last lane of an odd count is discarded
      fz = f.z.y; fw = f.w.y; cz = c.z.y; cw = c.w.y;
      bad = lane_final<INTEG, COUPLED>(a.m, a.lv, a.offset + j + 1, fz, fw, cz, cw, my);
      o[4] = fz; o[5] = fw;
      o[6] = COUPLED ? cz : 0.0f;
      o[7] = COUPLED ? cw : 0.0f;
      a.flags[j + 1] = bad ? 1 : 0;
    }
#endif
  } else {
    const uint64_t j = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
    if (j >= a.N) return;
    Path<R> f, c;
    bool bad;
    run_pair<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, f, c, bad, NoTrace<R>());
    R* o = a.states + 4 * j;
    o[0] = f.z; o[1] = f.w;
    o[2] = COUPLED ? c.z : R(0);
    o[3] = COUPLED ? c.w : R(0);
    a.flags[j] = bad ? 1 : 0;
  }
}

template <int INTEG, typename R, bool COUPLED>
__global__ void __launch_bounds__(kBlock) k_trace(const __grid_constant__ PathsArgs<R> a) {
  const uint64_t j = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (j >= a.N) return;
  const int64_t M = a.lv.M;
  Trace<R> tr;
  tr.f = a.tf ? a.tf + (uint64_t)3 * (M + 1) * j : nullptr;
  tr.c = (COUPLED && a.tc) ? a.tc + (uint64_t)3 * (M / 2 + 1) * j : nullptr;
  tr.fh = a.thf ? a.thf + (uint64_t)3 * M * j : nullptr;
  tr.ch = (COUPLED && a.thc) ? a.thc + (uint64_t)3 * (M / 2) * j : nullptr;
  Path<R> f, c;
  bool bad;
  run_pair_exact<INTEG, R, COUPLED>(a.m, a.lv, a.offset + j, f, c, bad, tr);
}

// ---------------------------------------------------------------------------
// Dispatch helpers
// ---------------------------------------------------------------------------
template <typename R, template <int, typename, bool> class K, typename Args>
cudaError_t launch3(int integ, bool coupled, dim3 grid, const Args& args, cudaStream_t st) {
#define MLMC_LAUNCH(I)                                                        \
  if (coupled) K<I, R, true>::launch(grid, args, st);                          \
  else K<I, R, false>::launch(grid, args, st);
  if (integ == kSE) { MLMC_LAUNCH(kSE) }
  else if (integ == kGL) { MLMC_LAUNCH(kGL) }
  else { MLMC_LAUNCH(kBAOAB) }
#undef MLMC_LAUNCH
  return cudaGetLastError();
}

template <int I, typename R, bool C>
struct SumsK {
  static void launch(dim3 g, const SumsArgs<R>& a, cudaStream_t st) {
    k_level_sums<I, R, C><<<g, kBlock, 0, st>>>(a);
  }
};
template <int I, typename R, bool C>
struct PathsK {
  static void launch(dim3 g, const PathsArgs<R>& a, cudaStream_t st) {
    k_paths<I, R, C><<<g, kBlock, 0, st>>>(a);
  }
};
template <int I, typename R, bool C>
struct PathsVK {
  static void launch(dim3 g, const PathsArgs<R>& a, cudaStream_t st) {
    k_paths_v<I, R, C><<<g, kBlock, 0, st>>>(a);
  }
};
template <int I, typename R, bool C>
struct TraceK {
  static void launch(dim3 g, const PathsArgs<R>& a, cudaStream_t st) {
    k_trace<I, R, C><<<g, kBlock, 0, st>>>(a);
  }
};

template <typename R>
cudaError_t level_sums_impl(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                            uint64_t offset, Partial* partials, int grid, cudaStream_t st) {
  SumsArgs<R> a;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.partials = partials;
  return launch3<R, SumsK>(integ, ls.coupled, dim3(grid), a, st);
}

template <typename R>
cudaError_t multilevel_impl(int integ, const HostModel& hm, const ReqPlan* plan, int n_req,
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
    a.req[r].single = plan[r].single;
  }
  a.n_req = n_req;
  a.n_items = n_items;
  a.partials = partials;
  a.counter = counter;
  if (integ == kSE) k_multilevel<kSE, R><<<grid, kBlock, 0, st>>>(a);
  else if (integ == kGL) k_multilevel<kGL, R><<<grid, kBlock, 0, st>>>(a);
  else k_multilevel<kBAOAB, R><<<grid, kBlock, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t pdf_impl(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                     uint64_t offset, int k, double* partials, int grid, cudaStream_t st);

template <typename R>
cudaError_t multilevel_dev_impl(int integ, const HostModel& hm, const DevPlan* plan,
                                Partial* partials, unsigned int* counter, int grid,
                                cudaStream_t st) {
  const Model<R> m = make_model<R>(hm);
  if (integ == kSE) k_multilevel_dev<kSE, R><<<grid, kBlock, 0, st>>>(m, plan, partials, counter);
  else if (integ == kGL) k_multilevel_dev<kGL, R><<<grid, kBlock, 0, st>>>(m, plan, partials, counter);
  else k_multilevel_dev<kBAOAB, R><<<grid, kBlock, 0, st>>>(m, plan, partials, counter);
  return cudaGetLastError();
}

template <typename R>
cudaError_t multilevel_table_impl(int integ, const void* models, size_t stride, const PlanReq* reqs,
                                  int n_req, uint32_t n_items, Partial* partials,
                                  unsigned int* counter, int grid, cudaStream_t st) {
  const char* mm = (const char*)models;
  if (integ == kSE)
    k_multilevel_table<kSE, R><<<grid, kBlock, 0, st>>>(mm, stride, reqs, n_req, n_items, partials,
                                                        counter);
  else if (integ == kGL)
    k_multilevel_table<kGL, R><<<grid, kBlock, 0, st>>>(mm, stride, reqs, n_req, n_items, partials,
                                                        counter);
  else
    k_multilevel_table<kBAOAB, R><<<grid, kBlock, 0, st>>>(mm, stride, reqs, n_req, n_items,
                                                           partials, counter);
  return cudaGetLastError();
}

template <typename R>
cudaError_t pdf_impl(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                     uint64_t offset, int k, double* partials, int grid, cudaStream_t st) {
  PdfArgs<R> a;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.k = k;
  a.binw = (R)(hm.H / (double)k);
  a.partials = partials;
  return launch3<R, PdfK>(integ, ls.coupled, dim3(grid), a, st);
}

template <typename R>
cudaError_t paths_impl(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                       uint64_t offset, void* states, int32_t* flags, void* tf, void* tc,
                       void* thf, void* thc, bool trace, cudaStream_t st) {
  PathsArgs<R> a;
  a.thf = (R*)thf;
  a.thc = (R*)thc;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.states = (R*)states;
  a.flags = flags;
  a.tf = (R*)tf;
  a.tc = (R*)tc;
  const dim3 g((unsigned)((N + kBlock - 1) / kBlock));
  if (N == 0) return cudaSuccess;
  if (trace) return launch3<R, TraceK>(integ, ls.coupled, g, a, st);
  return launch3<R, PathsK>(integ, ls.coupled, g, a, st);
}

template <typename R>
cudaError_t paths_variant_impl(int integ, const HostModel& hm, const LevelSpec& ls, uint64_t N,
                               uint64_t offset, void* states, int32_t* flags, cudaStream_t st) {
  PathsArgs<R> a;
  a.m = make_model<R>(hm);
  a.lv = make_level<R>(ls);
  a.N = N;
  a.offset = offset;
  a.states = (R*)states;
  a.flags = flags;
  a.tf = nullptr;
  a.tc = nullptr;
  a.thf = nullptr;
  a.thc = nullptr;
  if (N == 0) return cudaSuccess;
  const uint64_t per_block = (MLMC_X2 && std::is_same<R, float>::value) ? 2 * kBlock : kBlock;
  const dim3 g((unsigned)((N + per_block - 1) / per_block));
  return launch3<R, PathsVK>(integ, ls.coupled, g, a, st);
}

template <typename R>
int blocks_per_sm_impl(int integ, bool multilevel) {
  int nb = 0;
  cudaError_t e;
  if (multilevel) {
    if (integ == kSE) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_multilevel<kSE, R>, kBlock, 0);
    else if (integ == kGL) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_multilevel<kGL, R>, kBlock, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_multilevel<kBAOAB, R>, kBlock, 0);
  } else {
    if (integ == kSE) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level_sums<kSE, R, true>, kBlock, 0);
    else if (integ == kGL) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level_sums<kGL, R, true>, kBlock, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_level_sums<kBAOAB, R, true>, kBlock, 0);
  }
  if (e != cudaSuccess || nb < 1) nb = 1;
  if (nb > kMaxBlocksPerSM) nb = kMaxBlocksPerSM;
  return nb;
}

}  // namespace MLMC_KNS
}  // namespace mlmc
