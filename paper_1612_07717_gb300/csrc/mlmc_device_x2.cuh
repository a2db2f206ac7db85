// mlmc_device_x2.cuh -- two FP32 path pairs per thread on the packed FP32
// pipe of sm_103a (FFMA2 / FMUL2 / FADD2 through __ffma2_rn, __fmul2_rn,
// __fadd2_rn).
//
// The path kernel is issue-bound: about half of its instructions are FP32
// multiplies and adds.  Running two independent path pairs in the two lanes
// of a float2 issues each of those once for both paths; the SFU operations,
// compares, selects, min/max and the Philox integer rounds stay per lane.
// Every lane performs exactly the operations of the scalar code in
// mlmc_device.cuh, in the same order and rounding, so a path computed here is
// bit-identical to the same path computed one per thread: negations are
// folded into constants (nlam = -lambda, -h log2 e) instead of applied to a
// packed operand, and each scalar fma(a, b, c) stays a fused operation.
//
// References are to Katsiolides et al., arXiv 1612.07717.
#pragma once
#include "mlmc_device.cuh"


namespace mlmc {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(ptx_rsqrt(a.x), ptx_rsqrt(a.y)); }
__device__ __forceinline__ float2 sel2(bool px, bool py, float2 a, float2 b) {
  return make_float2(px ? a.x : b.x, py ? a.y : b.y);
}

// Loop constants of a level as lane pairs (kept in registers across steps).
struct LevelX2 {
  float2 h, h2, hc, hc2;
  float2 hl2, hcl2;               // h log2 e (fine and coarse)
  float2 h2x, hc2x;               // -2h and -4h: the SE noise variance factor of each step
};

__device__ __forceinline__ LevelX2 make_level_x2(const Level<float>& lv) {
  LevelX2 k;
  k.h = f2(lv.h); k.h2 = f2(lv.h2); k.hc = f2(lv.hc); k.hc2 = f2(lv.hc2);
  k.hl2 = f2(lv.hl2); k.hcl2 = f2(lv.hcl2);
  k.h2x = f2(-(2.0f * lv.h)); k.hc2x = f2(-(2.0f * lv.hc));
  return k;
}

// Profiles of mlmc_device.cuh's profile(), both lanes; returns -lambda (and
// -sigma_u when NSU).
template <bool NSU = false>
__device__ __forceinline__ void profile_x2(const Model<float>& m, float2 z, float2& sig_u,
                                           float2& nlam, float2& g0, float2& g1) {
  const float2 zc = make_float2(fminf(fmaxf(z.x, m.eps), m.Hme), fminf(fmaxf(z.y, m.eps), m.Hme));
  const bool ix = zc.x == z.x, iy = zc.y == z.y;
  const float2 s = fma2(zc, f2(-m.invH), f2(1.0f));
  const float2 t = rsqrt2(s);
  const float2 q = mul2(s, t);
  const float2 s34 = mul2(q, rsqrt2(t));
  sig_u = mul2(f2(NSU ? -m.A : m.A), s34);
  const float2 rz = make_float2(ptx_rcp(zc.x), ptx_rcp(zc.y));
  nlam = mul2(mul2(f2(-m.Akt), s34), add2(rz, f2(m.cfu)));
  g0 = mul2(sel2(ix, iy, f2(m.hD), f2(m.hD_out)), q);
  g1 = mul2(sel2(ix, iy, f2(m.hDs), f2(m.hDs_out)), mul2(t, t));
}

__device__ __forceinline__ void drift_coef_x2(const Model<float>& m, float2 z, float2& g0,
                                              float2& g1) {
  const float2 zc = make_float2(fminf(fmaxf(z.x, m.eps), m.Hme), fminf(fmaxf(z.y, m.eps), m.Hme));
  const bool ix = zc.x == z.x, iy = zc.y == z.y;
  const float2 s = fma2(zc, f2(-m.invH), f2(1.0f));
  const float2 t = rsqrt2(s);
  g0 = mul2(sel2(ix, iy, f2(m.hD), f2(m.hD_out)), mul2(s, t));
  g1 = mul2(sel2(ix, iy, f2(m.hDs), f2(m.hDs_out)), mul2(t, t));
}

// O-step factors (ou_factors / exp_pair of mlmc_device.cuh) from -lambda,
// with the signs carried instead of applied (a packed operand cannot be
// negated for free): ny = nlam (h log2 e) = -y, nsu = -sigma_u and
// nom = -(1 - e^2), from nseries = s ny and ndirect = e e - 1.  Round to
// nearest is symmetric, so c = nsu (nom rsqrt(-nom)) has exactly the bits of
// su (om rsqrt(om)), and ny > -0.07 is the test y < 0.07.
__device__ __forceinline__ void ou_factors_x2(float2 nsu, float2 nlam, float2 hl2, float2& e,
                                              float2& c) {
  const float2 ny = mul2(nlam, hl2);
  e = make_float2(ptx_ex2(ny.x), ptx_ex2(ny.y));
  const float a = 2.0f * kLn2;
  // The series runs per lane on scalar FFMA, which the lighter FMA pipe can
  // take: the packed ops keep the heavy FMA pipe busiest, and moving this
  // chain off it was measured faster (0.8 %), while moving more was slower.
  const float c5 = a * a * a * a * a / 120.0f, c4 = a * a * a * a / 24.0f;
  const float c3 = a * a * a / 6.0f, c2 = a * a / 2.0f;
  const float sx = fmaf(fmaf(fmaf(fmaf(c5, ny.x, c4), ny.x, c3), ny.x, c2), ny.x, a);
  const float sy = fmaf(fmaf(fmaf(fmaf(c5, ny.y, c4), ny.y, c3), ny.y, c2), ny.y, a);
  const float2 nseries = make_float2(sx * ny.x, sy * ny.y);
  const float2 ndirect = fma2(e, e, f2(-1.0f));
  const float2 nom = sel2(ny.x > -0.07f, ny.y > -0.07f, nseries, ndirect);
  c = mul2(nsu, mul2(nom, make_float2(ptx_rsqrt(-nom.x), ptx_rsqrt(-nom.y))));
}

// Box-Muller of mlmc_device.cuh on two word pairs (lane x: path a, lane y:
// path b).  -r = (2 ln 2 log2 u_a) rsqrt(-2 ln 2 log2 u_a), exactly the
// negation of the scalar r.
__device__ __forceinline__ void box_muller_x2(uint32_t xa0, uint32_t xa1, uint32_t xb0,
                                              uint32_t xb1, float2& na, float2& nb) {
  const float k1 = 0.99999994039535522461f;
  const float2 ua = add2(make_float2(__uint_as_float((xa0 >> 9) | 0x3F800000u),
                                     __uint_as_float((xa1 >> 9) | 0x3F800000u)), f2(-k1));
  const float2 ub = add2(make_float2(__uint_as_float((xb0 >> 9) | 0x3F800000u),
                                     __uint_as_float((xb1 >> 9) | 0x3F800000u)), f2(-k1));
  const float2 ns2 = mul2(f2(2.0f * kLn2), make_float2(ptx_lg2(ua.x), ptx_lg2(ua.y)));
  const float2 nr = mul2(ns2, make_float2(ptx_rsqrt(-ns2.x), ptx_rsqrt(-ns2.y)));
  const float2 t = mul2(f2(6.28318530717958647692f), add2(ub, f2(-0.5f)));
  na = mul2(nr, make_float2(ptx_cos(t.x), ptx_cos(t.y)));
  nb = mul2(nr, make_float2(ptx_sin(t.x), ptx_sin(t.y)));
}

// Path state of two paths.
struct PathX2 {
  float2 z, w, S, g0, g1;
  float2 wm;
};

// reflect_fast of mlmc_device.cuh per lane (its min/abs forms have no
// packed equivalent).
__device__ __forceinline__ void reflect_x2(const Model<float>& m, PathX2& p) {
  const float zax = fabsf(p.z.x), zay = fabsf(p.z.y);
  const float rx = fminf(zax, m.twoH - zax), ry = fminf(zay, m.twoH - zay);
  const bool fx = rx != p.z.x, fy = ry != p.z.y;
  p.w = make_float2(fx ? -p.w.x : p.w.x, fy ? -p.w.y : p.w.y);
  p.S = make_float2(fx ? -p.S.x : p.S.x, fy ? -p.S.y : p.S.y);
  p.z = make_float2(rx, ry);
}

__device__ __forceinline__ void track_wm(PathX2& p) {
  p.wm = make_float2(fmaxf(p.wm.x, fabsf(p.w.x)), fmaxf(p.wm.y, fabsf(p.w.y)));
}

// se_step: acc = fma(-lambda, w, fma(g1 w, w, g0)); amp = sigma_w sqrt(2 h lambda)
// with 2 h lambda = (-2h)(-lambda).
__device__ __forceinline__ void se_step_x2(const Model<float>& m, float2 h, float2 m2h, PathX2& p,
                                           float2 xi) {
  float2 su, nlam, g0, g1;
  profile_x2(m, p.z, su, nlam, g0, g1);
  const float2 v = mul2(m2h, nlam);
  const float2 amp = mul2(su, mul2(v, rsqrt2(v)));
  const float2 acc = fma2(nlam, p.w, fma2(mul2(g1, p.w), p.w, g0));
  p.w = fma2(amp, xi, fma2(h, acc, p.w));
  track_wm(p);
  p.z = fma2(p.w, h, p.z);
  reflect_x2(m, p);
}

__device__ __forceinline__ float2 gl_step_x2(const Model<float>& m, float2 h, float2 hl2,
                                             PathX2& p, float2 xi) {
  float2 nsu, nlam, g0, g1, e, c;
  profile_x2<true>(m, p.z, nsu, nlam, g0, g1);
  ou_factors_x2(nsu, nlam, hl2, e, c);
  const float2 us = fma2(c, xi, mul2(e, p.w));
  p.w = fma2(h, fma2(mul2(g1, us), us, g0), us);
  track_wm(p);
  p.z = fma2(p.w, h, p.z);
  reflect_x2(m, p);
  return e;
}

__device__ __forceinline__ void baoab_pre_x2(const Model<float>& m, float2 h2, PathX2& p) {
  p.w = fma2(h2, fma2(mul2(p.g1, p.w), p.w, p.g0), p.w);
  track_wm(p);
  p.z = fma2(p.w, h2, p.z);
  reflect_x2(m, p);
}

__device__ __forceinline__ float2 baoab_post_x2(const Model<float>& m, float2 hl2, float2 h2,
                                                PathX2& p, float2 xi) {
  float2 nsu, nlam, g0, g1, e, c;
  profile_x2<true>(m, p.z, nsu, nlam, g0, g1);
  ou_factors_x2(nsu, nlam, hl2, e, c);
  p.w = fma2(c, xi, mul2(e, p.w));
  track_wm(p);
  p.z = fma2(p.w, h2, p.z);
  reflect_x2(m, p);
  drift_coef_x2(m, p.z, p.g0, p.g1);
  p.w = fma2(h2, fma2(mul2(p.g1, p.w), p.w, p.g0), p.w);
  return e;
}

template <int INTEG>
__device__ __forceinline__ void fine_step_x2(const Model<float>& m, const LevelX2& k, PathX2& p,
                                             float2 xi, float2& Sn, float2& e) {
  if (INTEG == kSE) {
    Sn = p.S;
    e = f2(0.0f);
    se_step_x2(m, k.h, k.h2x, p, xi);
  } else if (INTEG == kGL) {
    Sn = p.S;
    e = gl_step_x2(m, k.h, k.hl2, p, xi);
  } else {
    baoab_pre_x2(m, k.h2, p);
    Sn = p.S;
    e = baoab_post_x2(m, k.hl2, k.h2, p, xi);
  }
}

// coarse_step of mlmc_device.cuh (the coupling of Sections 3.3 and 4.1) on both lanes.
template <int INTEG>
__device__ __forceinline__ void coarse_step_x2(const Model<float>& m, const LevelX2& k, PathX2& p,
                                               float2 xa, float2 xb, float2 Sa, float2 Sb,
                                               float2 ea) {
  if (m.coupling) { Sa = f2(1.0f); Sb = f2(1.0f); }
  if (INTEG == kSE) {
    const float2 Sc = m.coupling ? f2(1.0f) : p.S;
    const float2 xc = mul2(mul2(Sc, f2(0.70710678118654752440f)), fma2(Sa, xa, mul2(Sb, xb)));
    se_step_x2(m, k.hc, k.hc2x, p, xc);
  } else if (INTEG == kGL) {
    const float2 Sc = m.coupling ? f2(1.0f) : p.S;
    const float2 xc = mul2(mul2(Sc, rsqrt2(fma2(ea, ea, f2(1.0f)))),
                           fma2(mul2(ea, Sa), xa, mul2(Sb, xb)));
    gl_step_x2(m, k.hc, k.hcl2, p, xc);
  } else {
    baoab_pre_x2(m, k.hc2, p);
    const float2 Sc = m.coupling ? f2(1.0f) : p.S;
    const float2 xc = mul2(mul2(Sc, rsqrt2(fma2(ea, ea, f2(1.0f)))),
                           fma2(mul2(ea, Sa), xa, mul2(Sb, xb)));
    baoab_post_x2(m, k.hcl2, k.hc2, p, xc);
  }
}

// What the start of every pair shares when z0 is fixed (w0 modes 0 and 1):
// sigma_u(z0) for the initial velocity and the BAOAB drift coefficients at
// z0.  Computed once per work item by the operations initial_state and
// drift_coef_x2 perform for each pair, so the start values keep their bits.
struct StartX2 {
  float su0;
  float2 g0, g1;
};

__device__ __forceinline__ StartX2 start_x2(const Model<float>& m) {
  StartX2 s;
  float lam, g0, g1;
  profile(m, m.z0, s.su0, lam, g0, g1);
  drift_coef_x2(m, f2(m.z0), s.g0, s.g1);
  return s;
}

// Path pairs i and i + 1 of a level, fast reflection; flag_x / flag_y report
// a lane that needs the exact replay (see reflect_fast).
template <int INTEG, bool COUPLED>
__device__ __forceinline__ void run_pair_x2_fast(const Model<float>& m, const Level<float>& lv,
                                                 const StartX2& s0, uint64_t i, PathX2& f,
                                                 PathX2& c, bool& flx, bool& fly) {
  const uint64_t i1 = i + 1;
  const uint32_t alo = (uint32_t)i, ahi = (uint32_t)(i >> 32);
  const uint32_t blo = (uint32_t)i1, bhi = (uint32_t)(i1 >> 32);
  const uint32_t aw2 = ahi ^ lv.c2, bw2 = bhi ^ lv.c2;
  f.S = f2(1.0f);
  f.g0 = f2(0.0f);
  f.g1 = f2(0.0f);
  f.wm = f2(0.0f);
  if (m.w0_mode == 2) {  // well mixed: each pair draws its own height
    float za, wa, zb, wb;
    initial_state(m, lv, alo, ahi, za, wa);
    initial_state(m, lv, blo, bhi, zb, wb);
    f.z = make_float2(za, zb);
    f.w = make_float2(wa, wb);
    if (INTEG == kBAOAB) drift_coef_x2(m, f.z, f.g0, f.g1);
  } else {
    f.z = f2(m.z0);
    f.w = f2(m.w0);
    if (m.w0_mode == 1) {  // initial_state's draw from the reserved block
      const uint4 xa = philox10(m.rk0, m.rk1, 0xFFFFFFFFu, alo, aw2, m.stream_id);
      const uint4 xb = philox10(m.rk0, m.rk1, 0xFFFFFFFFu, blo, bw2, m.stream_id);
      float na, nb, unused;
      box_muller(xa.x, xa.y, na, unused);
      box_muller(xb.x, xb.y, nb, unused);
      f.w = make_float2(s0.su0 * na, s0.su0 * nb);
    }
    if (INTEG == kBAOAB) { f.g0 = s0.g0; f.g1 = s0.g1; }
  }
  c = f;
  const LevelX2 k = make_level_x2(lv);
  const int64_t M = lv.M;
  const uint32_t nblk = (uint32_t)(M >> 2);
  float2 Sa, Sb, ea, eb;
  for (uint32_t b = 0; b < nblk; ++b) {
    const uint4 xa = philox10(m.rk0, m.rk1, b, alo, aw2, m.stream_id);
    const uint4 xb = philox10(m.rk0, m.rk1, b, blo, bw2, m.stream_id);
    float2 xi0, xi1, xi2, xi3;
    box_muller_x2(xa.x, xb.x, xa.y, xb.y, xi0, xi1);
    box_muller_x2(xa.z, xb.z, xa.w, xb.w, xi2, xi3);
    if (COUPLED) {
      fine_step_x2<INTEG>(m, k, f, xi0, Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi1, Sb, eb);
      coarse_step_x2<INTEG>(m, k, c, xi0, xi1, Sa, Sb, ea);
      fine_step_x2<INTEG>(m, k, f, xi2, Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi3, Sb, eb);
      coarse_step_x2<INTEG>(m, k, c, xi2, xi3, Sa, Sb, ea);
    } else {
      fine_step_x2<INTEG>(m, k, f, xi0, Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi1, Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi2, Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi3, Sa, ea);
    }
  }
  const int tail = (int)(M & 3);
  if (tail) {
    const uint4 xa = philox10(m.rk0, m.rk1, nblk, alo, aw2, m.stream_id);
    const uint4 xb = philox10(m.rk0, m.rk1, nblk, blo, bw2, m.stream_id);
    float2 xi[4];
    box_muller_x2(xa.x, xb.x, xa.y, xb.y, xi[0], xi[1]);
    box_muller_x2(xa.z, xb.z, xa.w, xb.w, xi[2], xi[3]);
    if (COUPLED) {
      fine_step_x2<INTEG>(m, k, f, xi[0], Sa, ea);
      fine_step_x2<INTEG>(m, k, f, xi[1], Sb, eb);
      coarse_step_x2<INTEG>(m, k, c, xi[0], xi[1], Sa, Sb, ea);
    } else {
      for (int j = 0; j < tail; ++j) fine_step_x2<INTEG>(m, k, f, xi[j], Sa, ea);
    }
  }
  const float hA = INTEG == kBAOAB ? lv.h2 : lv.h;
  const float hAc = INTEG == kBAOAB ? lv.hc2 : lv.hc;
  flx = f.wm.x * hA > m.H;
  fly = f.wm.y * hA > m.H;
  if (COUPLED) {
    flx |= c.wm.x * hAc > m.H;
    fly |= c.wm.y * hAc > m.H;
  }
}

}  // namespace mlmc
