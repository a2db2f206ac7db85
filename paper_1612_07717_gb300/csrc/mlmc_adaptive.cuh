// mlmc_adaptive.cuh -- adaptive, non-nested timesteps for SE and GL
// (Section 7.2 of Katsiolides et al., arXiv 1612.07717), device side.
//
// Step rule, Eq. (adaptive h): h_n = min(h, lambda(X_adapt) / lambda(X_n) h)
// with X_n the stepping path's own position at the start of its step.
// lambda decreases with height, so the ratio is below 1 exactly when the
// clamped X_n lies below X_adapt; the step is then floor(1024 ratio) / 1024
// of h (at least 1/1024 by the parameter check): the same rule on every
// level and never longer than the paper's step.  Time runs in integer units
// of h_l / 1024 (32 bits): a fine step is at most 1024 units, a coarse one
// 2048, T is 1024 M_l, the last step of a path ends exactly at T, and fine
// and coarse time points of a pair are compared exactly.
//
// Coupling on the merged grid: interval j between consecutive fine or
// coarse time points carries the normal xi_j (element j mod 4 of Philox
// block j / 4, the counter of fine step j on a uniform grid).  Each path
// accumulates, for the intervals inside its current step,
//   SE (Eq. AdaptivityIncrementEuler):
//     A += S_j^(f) sigma sqrt(d_j) xi_j
//   GL (Eq. AdaptivityIncrementSplitting, applied recursively):
//     A  = A e^{-lambda d_j} + S_j^(f) sigma sqrt((1 - e^{-2 lambda d_j}) / (2 lambda)) xi_j
// with sigma = sigma_w sqrt(2 lambda), lambda the path's own lambda at the
// start of the step and the parities dropped on the fine path; the step
// then uses S_i^(c) A (fine path: A) in place of sigma sqrt(h) xi (SE) or of
// the O-step noise (GL).
//
// Work runs in rounds: a round draws one Philox block (four normals) for
// every lane at once and iterates until the lane has used them; one
// iteration finishes exactly one step, that of the path the pair keeps first
// (the one whose step ends first, the fine one when both end at the same
// tick), in place, so every lane of a warp runs the same step code whichever
// path it advances and no path state is copied unless the order changes.  A thread runs its pairs back to back (a finished pair
// is replaced at the next round), so a lane with short pairs does not wait
// for a warp-mate's long one; its pairs still enter its sums in index order.
#pragma once
#include "mlmc_device.cuh"

namespace mlmc {

constexpr uint32_t kNoStep = 0xFFFFFFFFu;  // t_end of a path that has reached T

template <typename R>
struct APath {
  R z, w, S;
  R su, lam, g0, g1;  // profile at the start of the current step
  R h;                // length of the current step [s]
  R A;                // sigma times the noise increment accumulated so far
  R E;                // GL: exp(-lambda x the part of the step accumulated so far)
  uint32_t t_end;     // unit at which the current step ends
};

__device__ __forceinline__ float adiv(float a, float b) { return a * ptx_rcp(b); }
__device__ __forceinline__ double adiv(double a, double b) { return a / b; }

// Start a step of a path at unit t: the profile at X_n, the step rule, the
// cap at T.  scale: 1 for the fine path, 2 for the coarse one (its h is 2048
// units); usec: seconds per unit.
template <typename R>
__device__ __forceinline__ void astep_begin(const Model<R>& m, APath<R>& p, uint32_t scale,
                                            uint32_t t, uint32_t T_units, R usec) {
  profile(m, p.z, p.su, p.lam, p.g0, p.g1);
  const R zc = fmin_(fmax_(p.z, m.eps), m.Hme);
  uint32_t k = 1024u;
  if (zc < m.za) {
    k = (uint32_t)(R(1024) * adiv(m.lam_a, p.lam));  // floor of a positive value
    k = k < 1u ? 1u : (k > 1024u ? 1024u : k);
  }
  uint32_t n = k * scale;
  const uint32_t left = T_units - t;
  n = n < left ? n : left;
  p.h = (R)n * usec;
  p.t_end = t + n;
  p.A = R(0);
  p.E = R(1);
}

// Add an interval of d seconds with normal xi and parity weight wgt.  An
// empty interval (d = 0, wgt = 0) leaves the path unchanged: e = 2^0 = 1 and
// the square root's argument is kept positive (the floor is far below any
// real interval's 2 lambda d or 1 - e^2), so its product with wgt = 0 is 0.
template <int INTEG, typename R>
__device__ __forceinline__ void accumulate(APath<R>& p, R d, R xi, R wgt) {
  const R tiny = R(1e-30);
  if (INTEG == kSE) {
    p.A = fma(wgt * (p.su * sqrt_(fmax_((R(2) * p.lam) * d, tiny))), xi, p.A);
  } else {
    R e, om;
    exp_pair(p.lam * (d * R(1.4426950408889634074)), e, om);
    p.A = fma(wgt * (p.su * sqrt_(fmax_(om, tiny))), xi, p.A * e);
    p.E *= e;
  }
}

// Finish the current step with noise Sx A, then fold into [0, H].
template <int INTEG, typename R>
__device__ __forceinline__ void astep_finish(const Model<R>& m, APath<R>& p, R Sx, bool& bad) {
  if (INTEG == kSE) {
    const R acc = fma(-p.lam, p.w, fma(p.g1 * p.w, p.w, p.g0));
    p.w = fma(Sx, p.A, fma(p.h, acc, p.w));
  } else {
    const R us = fma(Sx, p.A, p.E * p.w);             // O
    p.w = fma(p.h, fma(p.g1 * us, us, p.g0), us);     // B at (X_n, U*)
  }
  p.z = fma(p.w, p.h, p.z);                           // A
  reflect_exact(m, p.z, p.w, p.S, bad);
}

// State of one pair between rounds: the path that ends its step first
// (the fine one when both end together) is kept in `a`, the other in `b`,
// so an iteration steps `a` in place and the pair only swaps when the order
// changes.
template <typename R>
struct APair {
  APath<R> a, b;
  bool a_fine;       // a holds the fine path
  uint32_t t;        // current unit (end of the last merged interval)
  uint32_t T_units;  // T in units of h_l / 1024
  uint32_t cap;      // iteration bound of the pair
  uint32_t it;       // iterations so far: one per step of either path
  uint32_t i_lo, w2; // counter words of the pair
  uint32_t j;        // merged intervals consumed (a multiple of 4 between rounds)
  uint32_t nf, nc;   // steps taken by the fine and the coarse path
  R usec;            // seconds per unit
  bool bad;
};

template <typename R>
__device__ __forceinline__ void apair_order(APair<R>& P) {
  const bool sw = P.b.t_end < P.a.t_end || (P.b.t_end == P.a.t_end && !P.a_fine);
  if (sw) {
    const APath<R> x = P.a;
    P.a = P.b;
    P.b = x;
    P.a_fine = !P.a_fine;
  }
}

// Start pair i of a level: the shared initial state and the first steps.
template <typename R, bool COUPLED>
__device__ __forceinline__ void apair_init(const Model<R>& m, const Level<R>& lv, uint64_t i,
                                           APair<R>& P) {
  P.i_lo = (uint32_t)i;
  const uint32_t i_hi = (uint32_t)(i >> 32);
  P.w2 = i_hi ^ lv.c2;
  P.T_units = (uint32_t)lv.M << 10;
  P.usec = lv.h * R(0.0009765625);
  R z0, w0;
  initial_state(m, lv, P.i_lo, i_hi, z0, w0);
  P.a.z = z0; P.a.w = w0; P.a.S = R(1);
  astep_begin(m, P.a, 1u, 0u, P.T_units, P.usec);
  P.b = P.a;
  if (COUPLED) astep_begin(m, P.b, 2u, 0u, P.T_units, P.usec);
  else P.b.t_end = kNoStep;
  P.a_fine = true;
  apair_order(P);
  // every step is at least one unit: at most T_units steps per path
  P.cap = 2u * P.T_units + 64u;
  P.it = 0;
  P.nf = 0;
  P.nc = 0;
  P.t = 0;
  P.j = 0;
  P.bad = false;
}

template <typename R>
__device__ __forceinline__ bool apair_done(const APair<R>& P) {
  return P.bad || P.a.t_end == kNoStep;
}

template <typename R> __device__ __forceinline__ R apair_zf(const APair<R>& P) { return P.a_fine ? P.a.z : P.b.z; }
template <typename R> __device__ __forceinline__ R apair_wf(const APair<R>& P) { return P.a_fine ? P.a.w : P.b.w; }
template <typename R> __device__ __forceinline__ R apair_zc(const APair<R>& P) { return P.a_fine ? P.b.z : P.a.z; }
template <typename R> __device__ __forceinline__ R apair_wc(const APair<R>& P) { return P.a_fine ? P.b.w : P.a.w; }

// One round: the four normals of Philox block j / 4, then iterations until
// they are used or the pair is done.  Each iteration adds the merged interval
// [t, tn] (if not empty) to both paths and finishes exactly one step, that of
// `a` (the fine one first when both end at tn).
template <int INTEG, typename R, bool COUPLED>
__device__ __forceinline__ void apair_round(const Model<R>& m, APair<R>& P) {
  const uint4 x = philox10(m.rk0, m.rk1, P.j >> 2, P.i_lo, P.w2, m.stream_id);
  R x0, x1, x2, x3;
  box_muller(x.x, x.y, x0, x1);
  box_muller(x.z, x.w, x2, x3);
  uint32_t q = 0;
  while (q < 4u) {
    const uint32_t tn = P.a.t_end;
    if (tn == kNoStep) break;
    if (P.it >= P.cap) { P.bad = true; break; }
    P.it += 1;
    const bool iv = tn > P.t;
    const R xi = q == 0 ? x0 : (q == 1 ? x1 : (q == 2 ? x2 : x3));
    const R d = (R)(tn - P.t) * P.usec;
    const bool fine = P.a_fine;
    const R Sf = fine ? P.a.S : P.b.S;                              // S_j^(f)
    const R wc = m.coupling ? R(1) : Sf;
    accumulate<INTEG>(P.a, d, xi, iv ? (fine ? R(1) : wc) : R(0));
    if (COUPLED) accumulate<INTEG>(P.b, d, xi, iv ? (fine ? wc : R(1)) : R(0));
    q += iv ? 1u : 0u;
    P.t = tn;
    P.nf += fine ? 1u : 0u;
    P.nc += fine ? 0u : 1u;
    const R Sx = (fine || m.coupling) ? R(1) : P.a.S;               // S_i^(c)
    astep_finish<INTEG>(m, P.a, Sx, P.bad);
    if (P.a.t_end == P.T_units) P.a.t_end = kNoStep;
    else astep_begin(m, P.a, fine ? 1u : 2u, P.t, P.T_units, P.usec);
    if (COUPLED) apair_order(P);
    if (P.bad) break;
  }
  P.j += 4;
}

template <typename R, bool COUPLED>
__device__ __forceinline__ void apair_finish(APair<R>& P) {
  P.bad |= !(isfinite(P.a.z) && isfinite(P.a.w));
  if (COUPLED) P.bad |= !(isfinite(P.b.z) && isfinite(P.b.w));
}

// One path pair of a level with adaptive timesteps (fine only when not
// COUPLED).  P.bad marks a diverged pair (or one past the step bound).
template <int INTEG, typename R, bool COUPLED>
__device__ __forceinline__ void run_pair_adapt(const Model<R>& m, const Level<R>& lv, uint64_t i,
                                               APair<R>& P) {
  apair_init<R, COUPLED>(m, lv, i, P);
  while (!apair_done(P)) apair_round<INTEG, R, COUPLED>(m, P);
  apair_finish<R, COUPLED>(P);
}

}  // namespace mlmc
