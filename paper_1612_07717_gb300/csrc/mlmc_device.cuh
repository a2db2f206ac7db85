// mlmc_device.cuh -- device-side model of the MLMC boundary-layer dispersion
// path for sm_103a: Philox4x32-10 normals, regularised profiles, the three
// integrators with elastic reflection, and the coupled fine/coarse pair.
//
// One path pair lives in registers of one thread; nothing here touches
// global memory except the optional trace writer.  R is float (the fast
// path) or double (the FP64 baseline).  The kernels are issue-bound, so the
// step code is written to keep the instruction count low: the reflection is
// branch-free, the O-step factors share one exponential, and the profile
// needs three SFU operations.
//
// References are to Katsiolides et al., arXiv 1612.07717.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

constexpr int kSE = 0, kGL = 1, kBAOAB = 2;

// ---------------------------------------------------------------------------
// Scenario constants, precomputed on the host for one parameter set.
// ---------------------------------------------------------------------------
template <typename R>
struct Model {
  R H, twoH, eps, Hme;  // depth, 2H, eps_reg, H - eps_reg
  R invH;               // 1 / H
  R A;                  // kappa_sigma u*                 (sigma_w = A s^{3/4})
  R Akt;                // A / kappa_tau                  (lambda = Akt s^{3/4} (1/z + c_f f/u*))
  R cfu;                // c_f f / u*
  R hD, hD_out;         // 1/2 d sigma_w^2/dz = hD s^{1/2} inside the band (hD_out outside)
  R hDs, hDs_out;       // 1/2 (d sigma_w^2/dz) / sigma_w^2 = hDs / s inside (hDs_out outside)
  R qthr;               // indicator threshold
  R z0, w0;             // release state
  R lim;                // 1e3 H: a path beyond it has diverged
  int32_t w0_mode, coupling;
  uint32_t stream_id;
  int32_t qoi1_mode;    // 0 indicator, 1 smoothed interval
  int32_t sdeg;         // degree of the smoothing polynomial (r + 1)
  R qa, qb, idelta;     // interval and 1 / delta of the smoothed QoI
  R pc[12];             // smoothing polynomial coefficients
  uint32_t rk0[10], rk1[10];  // Philox round keys of the seed
  // adaptive timesteps (Section 7.2)
  R za, lam_a;          // X_adapt and lambda(X_adapt)
};

// Per-level constants.
template <typename R>
struct Level {
  R h, h2;            // fine step h and h / 2
  R hc, hc2;          // coarse step 2h and h
  R hl2, hcl2;        // h log2(e) and 2h log2(e) (arguments of the base-2 exponential)
  int64_t M;          // fine steps
  uint32_t c2;        // level word xored into counter word 2: level << 24
  int32_t coupled;    // 0 on the coarsest level
};

// ---------------------------------------------------------------------------
// Precision-generic primitives.  Float: single SFU instructions through the
// PTX approximations with flush-to-zero (the kernels never see subnormal
// values that matter: the smallest is exp(-lambda h) underflowing to 0).
// Double: the IEEE routines.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ptx_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_rsqrt(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_sin(float x) {
  float r;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_cos(float x) {
  float r;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_(float x) { return ptx_rsqrt(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float rcp_(float x) { return ptx_rcp(x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float sqrt_(float x) { return x * ptx_rsqrt(x); }  // x > 0
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }

// O-step factors from y = lambda h log2(e) (the argument of the base-2
// exponential): e = exp(-lambda h) = 2^-y and 1 - e^2 = 1 - exp(-2 lambda h)
// without cancellation at small y.  Float: Taylor series of
// 1 - 2^{-2y} = 1 - e^{-2 y ln 2} through y^5 below y = 0.07 (truncation
// below 1.5e-8 relative), 1 - e*e above (cancellation below 5e-7 relative).
// Double: exp and expm1 of lambda h.
constexpr float kLn2 = 0.69314718055994530942f;
__device__ __forceinline__ void exp_pair(float y, float& e, float& om) {
  e = ptx_ex2(-y);
  const float a = 2.0f * kLn2;                       // 1 - e^{-a y} = a y - (a y)^2/2 + ...
  float s = a * a * a * a * a / 120.0f;
  s = fmaf(s, -y, a * a * a * a / 24.0f);
  s = fmaf(s, -y, a * a * a / 6.0f);
  s = fmaf(s, -y, a * a / 2.0f);
  s = fmaf(s, -y, a);
  const float series = s * y;
  const float direct = fmaf(-e, e, 1.0f);
  om = y < 0.07f ? series : direct;
}
__device__ __forceinline__ void exp_pair(double y, double& e, double& om) {
  const double x = y * 0.69314718055994530942;
  e = exp(-x);
  om = -expm1(-2.0 * x);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The round keys of the
// seed are precomputed on the host (they are the same for every thread).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(const uint32_t* __restrict__ rk0,
                                         const uint32_t* __restrict__ rk1, uint32_t c0,
                                         uint32_t c1, uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ rk0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ rk1[r];
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Uniform maps.  Float: u = (floor(x / 2^9) + 1/2) 2^-23, formed exactly by
// placing the top 23 bits in the mantissa of [1, 2) and subtracting
// 1 - 2^-24 (Sterbenz: exact).  Double: u = (x + 1/2) 2^-32, exact.
__device__ __forceinline__ float u01f(uint32_t x) {
  return __uint_as_float((x >> 9) | 0x3F800000u) - 0.99999994039535522461f;
}
__device__ __forceinline__ double u01d(uint32_t x) {
  return ((double)x + 0.5) * 2.3283064365386962890625e-10;
}

// Box-Muller on a word pair: R = sqrt(-2 ln u_a), angle 2 pi u_b.  The
// float path evaluates the angle as 2 pi (u_b - 1/2) in (-pi, pi), where the
// SFU sine and cosine are accurate, and negates (cos(t + pi) = -cos t);
// -2 ln u = -2 ln(2) log2(u).
__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, float& na, float& nb) {
  const float ua = u01f(xa), ub = u01f(xb);
  const float s2 = (-2.0f * kLn2) * ptx_lg2(ua);
  const float r = s2 * ptx_rsqrt(s2);
  const float t = 6.28318530717958647692f * (ub - 0.5f);
  na = -r * ptx_cos(t);
  nb = -r * ptx_sin(t);
}
__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, double& na, double& nb) {
  const double ua = u01d(xa), ub = u01d(xb);
  const double r = sqrt(-2.0 * log(ua));
  double sn, cs;
  sincospi(2.0 * ub, &sn, &cs);
  na = r * cs;
  nb = r * sn;
}
__device__ __forceinline__ float uni_(uint32_t x, float) { return u01f(x); }
__device__ __forceinline__ double uni_(uint32_t x, double) { return u01d(x); }

// ---------------------------------------------------------------------------
// Profiles, Eq. (profiles) with the cut-off of Eq. (regularisation).  With
// z_c the clamped height, s = 1 - z_c / H and t = s^{-1/2}:
//   sigma_w = A s^{3/4} = A (s t) rsqrt(t)
//   lambda  = sigma_w (1 + c_f f z_c / u*) / (kappa_tau z_c)
//           = (A / kappa_tau) s^{3/4} (1 / z_c + c_f f / u*)
//   1/2 d sigma_w^2/dz               = -3/4 A^2 s^{1/2} / H = hD (s t)
//   1/2 (d sigma_w^2/dz) / sigma_w^2 = -3/4 / (H s)        = hDs t^2
// so the drift term -dV/dX = 1/2 (1 + w^2 / sigma_w^2) d sigma_w^2/dz is
// g0 + g1 w^2.  Outside the band (z_c != z) the derivative of the frozen
// profile is 0 (hD_out = hDs_out = 0) unless the frozen-value reading is
// selected.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void profile(const Model<R>& m, R z, R& sig_u, R& lam, R& g0, R& g1) {
  const R zc = fmin_(fmax_(z, m.eps), m.Hme);
  const bool inb = zc == z;
  const R s = fma(-zc, m.invH, R(1));
  const R t = rsqrt_(s);
  const R q = s * t;
  const R s34 = q * rsqrt_(t);
  sig_u = m.A * s34;
  lam = (m.Akt * s34) * (rcp_(zc) + m.cfu);
  g0 = (inb ? m.hD : m.hD_out) * q;
  g1 = (inb ? m.hDs : m.hDs_out) * (t * t);
}

// Only the drift coefficients (the B half-steps of BAOAB).
template <typename R>
__device__ __forceinline__ void drift_coef(const Model<R>& m, R z, R& g0, R& g1) {
  const R zc = fmin_(fmax_(z, m.eps), m.Hme);
  const bool inb = zc == z;
  const R s = fma(-zc, m.invH, R(1));
  const R t = rsqrt_(s);
  g0 = (inb ? m.hD : m.hD_out) * (s * t);
  g1 = (inb ? m.hDs : m.hDs_out) * (t * t);
}

// ---------------------------------------------------------------------------
// Smoothed indicator (Section 5.1, Eqs. gr and SmoothedIndicator):
// g_r(x) = 1 for x < -1, p_r(x) on [-1, 1], 0 for x > 1, and
// P^{r,delta}_{[a,b]}(z) = g_r((z - b) / delta) - g_r((z - a) / delta).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R g_smooth(const Model<R>& m, R x) {
  R v = m.pc[11];
  for (int k = 10; k >= 0; --k) v = fma(v, x, m.pc[k]);
  return x < R(-1) ? R(1) : (x > R(1) ? R(0) : v);
}
template <typename R>
__device__ __forceinline__ R smoothed_interval(const Model<R>& m, R z) {
  return g_smooth(m, (z - m.qb) * m.idelta) - g_smooth(m, (z - m.qa) * m.idelta);
}

// ---------------------------------------------------------------------------
// Elastic reflection (Section 4): z -> -z at the ground, z -> 2H - z at the
// top, w -> -w, and the parity S = (-1)^{n_refl} flips.
//
// reflect_fast: one reflection, branch-free and exact: z' = min(|z|, 2H - |z|)
// equals z inside [0, H], -z below, 2H - z above; a reflection happened iff
// z' != z.  It equals the oracle's fold whenever the unfolded z lies in
// [-H, 2H], which holds when the A-step displacement |w| h_A is at most H
// (z starts every A-step inside [0, H]).  The path keeps the largest |w|
// entering an A-step; if |w|max h_A > H the caller replays the whole path
// with reflect_exact.  (Such steps only occur on paths that are diverging.)
//
// reflect_exact: the loop of single reflections, as in the oracle, with
// |z| > 1e3 H (or NaN) marking the path as diverged.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void reflect_fast(const Model<R>& m, R& z, R& w, R& S) {
  const R za = fabs(z);
  const R zr = fmin_(za, m.twoH - za);
  const bool flip = zr != z;
  w = flip ? -w : w;
  S = flip ? -S : S;
  z = zr;
}

template <typename R>
__device__ __forceinline__ void reflect_exact(const Model<R>& m, R& z, R& w, R& S, bool& bad) {
  for (int it = 0; it < 2100 && (z < R(0) || z > m.H); ++it) {
    if (!(fabs(z) <= m.lim)) { bad = true; return; }
    z = (z < R(0)) ? -z : m.twoH - z;
    w = -w;
    S = -S;
  }
}

template <typename R, bool EXACT>
__device__ __forceinline__ void reflect(const Model<R>& m, R& z, R& w, R& S, bool& flag) {
  if (EXACT) reflect_exact(m, z, w, S, flag);
  else reflect_fast(m, z, w, S);
}

// ---------------------------------------------------------------------------
// One path: position, velocity, parity and (BAOAB) the cached drift terms
// at the current position.
// ---------------------------------------------------------------------------
template <typename R>
struct Path {
  R z, w, S;
  R g0, g1;
  R wm;     // largest |w| entering an A-step
};

// Symplectic Euler, Eq. (MethodSymplecticEuler):
//   w' = (1 - lambda h) w - dV/dX h + sigma sqrt(h) xi,  z' = z + w' h,
// with sigma sqrt(h) = sigma_w sqrt(2 lambda h).
template <typename R, bool EX>
__device__ __forceinline__ void se_step(const Model<R>& m, R h, Path<R>& p, bool& flag, R xi) {
  R su, lam, g0, g1;
  profile(m, p.z, su, lam, g0, g1);
  const R amp = su * sqrt_((R(2) * h) * lam);
  const R acc = fma(-lam, p.w, fma(g1 * p.w, p.w, g0));
  p.w = fma(amp, xi, fma(h, acc, p.w));
  p.wm = fmax_(p.wm, fabs(p.w));
  p.z = fma(p.w, h, p.z);
  reflect<R, EX>(m, p.z, p.w, p.S, flag);
}

// O-step factors: e = exp(-lambda h) and the noise amplitude
// sigma sqrt((1 - e^{-2 lambda h}) / (2 lambda)) = sigma_w sqrt(1 - e^2);
// hl2 = h log2(e).
template <typename R>
__device__ __forceinline__ void ou_factors(R su, R lam, R hl2, R& e, R& c) {
  R om;
  exp_pair(lam * hl2, e, om);
  c = su * sqrt_(om);
}

// Geometric Langevin (OBA), Eq. (MethodSymplecticEulerOU).  Returns e.
template <typename R, bool EX>
__device__ __forceinline__ R gl_step(const Model<R>& m, R h, R hl2, Path<R>& p, bool& flag, R xi) {
  R su, lam, g0, g1, e, c;
  profile(m, p.z, su, lam, g0, g1);
  ou_factors(su, lam, hl2, e, c);
  const R us = fma(c, xi, e * p.w);          // O
  p.w = fma(h, fma(g1 * us, us, g0), us);    // B at (z_n, u*)
  p.wm = fmax_(p.wm, fabs(p.w));
  p.z = fma(p.w, h, p.z);                    // A
  reflect<R, EX>(m, p.z, p.w, p.S, flag);
  return e;
}

// BAOAB, Eq. (MethodBAOAB), folded after each A half-step.  The step is split
// at the noise: baoab_pre runs B and A and leaves the parity of the O time in
// p.S; baoab_post runs O, A, B.  p.g0 / p.g1 hold the drift terms at p.z.
template <typename R, bool EX>
__device__ __forceinline__ void baoab_pre(const Model<R>& m, R h2, Path<R>& p, bool& flag) {
  p.w = fma(h2, fma(p.g1 * p.w, p.w, p.g0), p.w);  // B half-step at z_n
  p.wm = fmax_(p.wm, fabs(p.w));
  p.z = fma(p.w, h2, p.z);                          // A half-step
  reflect<R, EX>(m, p.z, p.w, p.S, flag);
}
template <typename R, bool EX>
__device__ __forceinline__ R baoab_post(const Model<R>& m, R hl2, R h2, Path<R>& p, bool& flag,
                                        R xi) {
  R su, lam, g0, g1, e, c;
  profile(m, p.z, su, lam, g0, g1);                 // at z_{n+1/2}
  ou_factors(su, lam, hl2, e, c);
  p.w = fma(c, xi, e * p.w);                        // O
  p.wm = fmax_(p.wm, fabs(p.w));
  p.z = fma(p.w, h2, p.z);                          // A half-step
  reflect<R, EX>(m, p.z, p.w, p.S, flag);
  drift_coef(m, p.z, p.g0, p.g1);                   // at z_{n+1}
  p.w = fma(h2, fma(p.g1 * p.w, p.w, p.g0), p.w);   // B half-step
  return e;
}

// Fine sub-step with normal xi; returns the parity at the noise time (Sn)
// and the O-step factor e (GL/BAOAB) used by the coarse coupling.
// tr.half_fine(n, p) sees BAOAB's state after the first half of fine step n.
template <int INTEG, typename R, bool EX, class TR>
__device__ __forceinline__ void fine_step(const Model<R>& m, const Level<R>& lv, Path<R>& p,
                                          bool& flag, R xi, R& Sn, R& e, const TR& tr,
                                          int64_t n) {
  if (INTEG == kSE) {
    Sn = p.S;
    e = R(0);
    se_step<R, EX>(m, lv.h, p, flag, xi);
  } else if (INTEG == kGL) {
    Sn = p.S;
    e = gl_step<R, EX>(m, lv.h, lv.hl2, p, flag, xi);
  } else {
    baoab_pre<R, EX>(m, lv.h2, p, flag);
    tr.half_fine(n, p);
    Sn = p.S;
    e = baoab_post<R, EX>(m, lv.hl2, lv.h2, p, flag, xi);
  }
}

// Coarse step of 2h driven by the fine normals xa, xb of sub-steps 2k and
// 2k+1 (parities Sa, Sb, O-factor ea of sub-step 2k):
//   SE:       xi_c = S_c (S_a xa + S_b xb) / sqrt(2)          Eq. (euler_coupled_treatment)
//   GL/BAOAB: xi_c = S_c (ea S_a xa + S_b xb) / sqrt(ea^2 + 1) Eq. (splitting_coupled_treatment)
// With coupling = 1 (naive) all parities are taken as 1.
template <int INTEG, typename R, bool EX, class TR>
__device__ __forceinline__ void coarse_step(const Model<R>& m, const Level<R>& lv, Path<R>& p,
                                            bool& flag, R xa, R xb, R Sa, R Sb, R ea,
                                            const TR& tr, int64_t k) {
  if (m.coupling) { Sa = R(1); Sb = R(1); }
  if (INTEG == kSE) {
    const R Sc = m.coupling ? R(1) : p.S;
    const R xc = (Sc * R(0.70710678118654752440)) * fma(Sa, xa, Sb * xb);
    se_step<R, EX>(m, lv.hc, p, flag, xc);
  } else if (INTEG == kGL) {
    const R Sc = m.coupling ? R(1) : p.S;
    const R xc = (Sc * rsqrt_(fma(ea, ea, R(1)))) * fma(ea * Sa, xa, Sb * xb);
    gl_step<R, EX>(m, lv.hc, lv.hcl2, p, flag, xc);
  } else {
    baoab_pre<R, EX>(m, lv.hc2, p, flag);
    tr.half_coarse(k, p);
    const R Sc = m.coupling ? R(1) : p.S;
    const R xc = (Sc * rsqrt_(fma(ea, ea, R(1)))) * fma(ea * Sa, xa, Sb * xb);
    baoab_post<R, EX>(m, lv.hcl2, lv.hc2, p, flag, xc);
  }
}

// ---------------------------------------------------------------------------
// Initial state (shared by the fine and coarse path): fixed, w0 ~
// N(0, sigma_w(z0)^2), or the well-mixed state; the draws come from the
// reserved counter block 0xFFFFFFFF.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void initial_state(const Model<R>& m, const Level<R>& lv, uint32_t i_lo,
                                              uint32_t i_hi, R& z, R& w) {
  z = m.z0;
  w = m.w0;
  if (m.w0_mode == 0) return;
  const uint4 x = philox10(m.rk0, m.rk1, 0xFFFFFFFFu, i_lo, i_hi ^ lv.c2, m.stream_id);
  R na, nb;
  box_muller(x.x, x.y, na, nb);
  if (m.w0_mode == 2) z = m.H * uni_(x.z, R(0));
  R su, lam, g0, g1;
  profile(m, z, su, lam, g0, g1);
  w = su * na;
}

// Trace sink: the production kernels pass NoTrace.
template <typename R>
struct NoTrace {
  __device__ __forceinline__ void fine(int64_t, const Path<R>&) const {}
  __device__ __forceinline__ void coarse(int64_t, const Path<R>&) const {}
  __device__ __forceinline__ void half_fine(int64_t, const Path<R>&) const {}
  __device__ __forceinline__ void half_coarse(int64_t, const Path<R>&) const {}
};
// Rows of (z, w, S): f / c after every step, fh / ch (BAOAB) after the
// first half of every step (the fold after its first A half-step); any of
// them may be null.
template <typename R>
struct Trace {
  R* f;   // (M+1) x 3
  R* c;   // (M/2+1) x 3
  R* fh;  // M x 3
  R* ch;  // M/2 x 3
  __device__ __forceinline__ static void put(R* t, int64_t row, const Path<R>& p) {
    if (t) { t[3 * row] = p.z; t[3 * row + 1] = p.w; t[3 * row + 2] = p.S; }
  }
  __device__ __forceinline__ void fine(int64_t row, const Path<R>& p) const { put(f, row, p); }
  __device__ __forceinline__ void coarse(int64_t row, const Path<R>& p) const { put(c, row, p); }
  __device__ __forceinline__ void half_fine(int64_t row, const Path<R>& p) const { put(fh, row, p); }
  __device__ __forceinline__ void half_coarse(int64_t row, const Path<R>& p) const { put(ch, row, p); }
};

// ---------------------------------------------------------------------------
// One path pair of a level (Section 3.3): fine path with M steps and, on
// coupled levels, the coarse path with M/2 steps driven by the same Brownian
// increments.  Normal n of the fine path is word n mod 4 of Philox block n/4.
// With EX = false the reflections are the fast single fold and `flag`
// reports a step that needed more (then the caller replays with EX = true);
// with EX = true `flag` is the diverged mark.
// ---------------------------------------------------------------------------
template <int INTEG, typename R, bool COUPLED, bool EX, class TR>
__device__ __forceinline__ void run_pair_impl(const Model<R>& m, const Level<R>& lv, uint64_t i,
                                              Path<R>& f, Path<R>& c, bool& flag, const TR& tr) {
  const uint32_t i_lo = (uint32_t)i, i_hi = (uint32_t)(i >> 32);
  const uint32_t w2 = i_hi ^ lv.c2;
  R z0, w0;
  initial_state(m, lv, i_lo, i_hi, z0, w0);
  f.z = z0; f.w = w0; f.S = R(1);
  f.g0 = R(0); f.g1 = R(0);
  f.wm = R(0);
  if (INTEG == kBAOAB) drift_coef(m, z0, f.g0, f.g1);
  c = f;
  flag = false;
  tr.fine(0, f);
  if (COUPLED) tr.coarse(0, c);
  const int64_t M = lv.M;
  const uint32_t nblk = (uint32_t)(M >> 2);
  R Sa, Sb, ea, eb;
  for (uint32_t b = 0; b < nblk; ++b) {
    const uint4 x = philox10(m.rk0, m.rk1, b, i_lo, w2, m.stream_id);
    R xi0, xi1, xi2, xi3;
    box_muller(x.x, x.y, xi0, xi1);
    box_muller(x.z, x.w, xi2, xi3);
    const int64_t n4 = 4 * (int64_t)b;
    if (COUPLED) {
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi0, Sa, ea, tr, n4);
      tr.fine(n4 + 1, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi1, Sb, eb, tr, n4 + 1);
      tr.fine(n4 + 2, f);
      coarse_step<INTEG, R, EX>(m, lv, c, flag, xi0, xi1, Sa, Sb, ea, tr, n4 / 2);
      tr.coarse(n4 / 2 + 1, c);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi2, Sa, ea, tr, n4 + 2);
      tr.fine(n4 + 3, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi3, Sb, eb, tr, n4 + 3);
      tr.fine(n4 + 4, f);
      coarse_step<INTEG, R, EX>(m, lv, c, flag, xi2, xi3, Sa, Sb, ea, tr, n4 / 2 + 1);
      tr.coarse(n4 / 2 + 2, c);
    } else {
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi0, Sa, ea, tr, n4);
      tr.fine(n4 + 1, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi1, Sa, ea, tr, n4 + 1);
      tr.fine(n4 + 2, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi2, Sa, ea, tr, n4 + 2);
      tr.fine(n4 + 3, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi3, Sa, ea, tr, n4 + 3);
      tr.fine(n4 + 4, f);
    }
  }
  const int tail = (int)(M & 3);  // fine steps left when M is not a multiple of 4
  if (tail) {
    const uint4 x = philox10(m.rk0, m.rk1, nblk, i_lo, w2, m.stream_id);
    R xi[4];
    box_muller(x.x, x.y, xi[0], xi[1]);
    box_muller(x.z, x.w, xi[2], xi[3]);
    const int64_t n0 = 4 * (int64_t)nblk;
    if (COUPLED) {
      // M even: tail is 2, one coarse step
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi[0], Sa, ea, tr, n0);
      tr.fine(n0 + 1, f);
      fine_step<INTEG, R, EX>(m, lv, f, flag, xi[1], Sb, eb, tr, n0 + 1);
      tr.fine(n0 + 2, f);
      coarse_step<INTEG, R, EX>(m, lv, c, flag, xi[0], xi[1], Sa, Sb, ea, tr, n0 / 2);
      tr.coarse(n0 / 2 + 1, c);
    } else {
      for (int j = 0; j < tail; ++j) {
        fine_step<INTEG, R, EX>(m, lv, f, flag, xi[j], Sa, ea, tr, n0 + j);
        tr.fine(n0 + j + 1, f);
      }
    }
  }
  if (!EX) {
    // a single fold per A-step is exact while |w| h_A <= H (see reflect_fast)
    const R hA = INTEG == kBAOAB ? lv.h2 : lv.h;
    const R hAc = INTEG == kBAOAB ? lv.hc2 : lv.hc;
    flag = f.wm * hA > m.H;
    if (COUPLED) flag |= c.wm * hAc > m.H;
  }
}

// A path pair with the diverged mark: the fast pass, replayed exactly (in
// the rare case a step crossed more than one layer depth).
template <int INTEG, typename R, bool COUPLED, class TR>
__device__ __forceinline__ void run_pair(const Model<R>& m, const Level<R>& lv, uint64_t i,
                                         Path<R>& f, Path<R>& c, bool& bad, const TR& tr) {
  bool multi;
  run_pair_impl<INTEG, R, COUPLED, false>(m, lv, i, f, c, multi, tr);
  bad = false;
  if (multi) run_pair_impl<INTEG, R, COUPLED, true>(m, lv, i, f, c, bad, tr);
  bad |= !(isfinite(f.z) && isfinite(f.w));
  if (COUPLED) bad |= !(isfinite(c.z) && isfinite(c.w));
}

// Always the exact reflection (trace output).
template <int INTEG, typename R, bool COUPLED, class TR>
__device__ __forceinline__ void run_pair_exact(const Model<R>& m, const Level<R>& lv, uint64_t i,
                                               Path<R>& f, Path<R>& c, bool& bad, const TR& tr) {
  run_pair_impl<INTEG, R, COUPLED, true>(m, lv, i, f, c, bad, tr);
  bad |= !(isfinite(f.z) && isfinite(f.w));
  if (COUPLED) bad |= !(isfinite(c.z) && isfinite(c.w));
}

}  // namespace mlmc
