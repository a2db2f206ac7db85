/*
 * oracle.c -- plain FP64 CPU restatement of the MLMC boundary-layer
 * dispersion method of arXiv 1612.07717.  TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the CPU-baseline leg of the benchmark are its
 * only users.  It shares no code with the CUDA library.
 *
 * The code follows the paper's notation: X is the particle height (z), U its
 * vertical velocity (w), S the reflection parity (-1)^{n_refl}, h the
 * timestep, xi a standard normal.  No blocking, fusion or reordering beyond
 * the equations as printed: every coefficient is evaluated from its
 * definition at the point where the equation asks for it.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread oracle.c -lm
 * (no FMA contraction, so x86 and Arm hosts give bit-identical results).
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror and Shaw,      */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11: ten rounds of a     */
/* multiply-hi/lo S-box on the counter, with a Weyl-sequence key schedule.   */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u; /* round multipliers        */
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u; /* golden ratio             */
static const uint32_t PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1              */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 32-bit word to a uniform in (0, 1); both maps are exact in FP64. */
static double uniform01(const orc_params* p, uint32_t x) {
  if (p->uniform_map == ORC_U23)
    return ((double)(x >> 9) + 0.5) * ldexp(1.0, -23);
  return ((double)x + 0.5) * ldexp(1.0, -32);
}

/* Philox words for (path i, level, counter block) of the query stream:
 * counter = (block, i_lo, i_hi xor (level << 24), stream_id), key = seed. */
static void philox_words(const orc_params* p, int level, uint64_t i, uint32_t block,
                         uint64_t seed, uint32_t x[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = block;
  ctr[1] = (uint32_t)(i & 0xFFFFFFFFu);
  ctr[2] = (uint32_t)(i >> 32) ^ ((uint32_t)level << 24);
  ctr[3] = p->stream_id;
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, x);
}

/* Box-Muller: a pair of uniforms to a pair of independent standard normals.
 * (The paper only asks for i.i.d. Normal(0,1) increments, after Eq.
 * MethodSymplecticEuler; this is the map both implementations share.) */
static void box_muller(double ua, double ub, double* xa, double* xb) {
  const double two_pi = 6.283185307179586476925286766559;
  double R = sqrt(-2.0 * log(ua));
  *xa = R * cos(two_pi * ub);
  *xb = R * sin(two_pi * ub);
}

void orc_normals4(const orc_params* p, int level, uint64_t i, uint32_t block,
                  uint64_t seed, double xi[4]) {
  uint32_t x[4];
  philox_words(p, level, i, block, seed, x);
  box_muller(uniform01(p, x[0]), uniform01(p, x[1]), &xi[0], &xi[1]);
  box_muller(uniform01(p, x[2]), uniform01(p, x[3]), &xi[2], &xi[3]);
}

/* ------------------------------------------------------------------------ */
/* Profiles, Eq. (profiles), with the hard cut-off of Eq. (regularisation)  */
/* and the optional Coriolis factor on tau.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double sigma_u;    /* sigma_U(X)                         */
  double sigma_u2;   /* sigma_U(X)^2                       */
  double dsig2_dX;   /* d sigma_U^2 / dX (regularised)      */
  double lambda;     /* 1 / tau(X)                          */
  double sigma;      /* sqrt(2 sigma_U^2 / tau)             */
} coef_t;

static coef_t coefficients(const orc_params* p, double X) {
  const double H = p->H;
  const double eps = p->eps_reg_frac * H;
  /* Eq. (regularisation): tau and sigma_U frozen outside [eps, H - eps]. */
  double Xc = X;
  if (Xc < eps) Xc = eps;
  if (Xc > H - eps) Xc = H - eps;
  coef_t c;
  c.sigma_u = p->kappa_sigma * p->u_star * pow(1.0 - Xc / H, 0.75);
  c.sigma_u2 = c.sigma_u * c.sigma_u;
  double tau = p->kappa_tau * Xc / c.sigma_u / (1.0 + p->c_f * p->f_coriolis * Xc / p->u_star);
  c.lambda = 1.0 / tau;
  c.sigma = sqrt(2.0 * c.sigma_u2 / tau);
  /* derivative of sigma_U^2 = (k u*)^2 (1 - X/H)^{3/2}; the regularised
   * profile is constant outside the band, so its derivative is 0 there. */
  const double ku2 = (p->kappa_sigma * p->u_star) * (p->kappa_sigma * p->u_star);
  int inside = (X >= eps) && (X <= H - eps);
  if (inside || p->drift_outside == 1)
    c.dsig2_dX = -1.5 * ku2 * sqrt(1.0 - Xc / H) / H;
  else
    c.dsig2_dX = 0.0;
  return c;
}

void orc_coefficients(const orc_params* p, double z, double out[5]) {
  coef_t c = coefficients(p, z);
  out[0] = c.sigma_u; out[1] = c.sigma_u2; out[2] = c.dsig2_dX;
  out[3] = c.lambda; out[4] = c.sigma;
}

/* dV/dX(X, U) = -1/2 (1 + U^2 / sigma_U^2) d sigma_U^2/dX, from the compact
 * form Eq. (generalisedsim) of Eq. (generalised). */
static double dVdX(const coef_t* c, double U) {
  return -0.5 * (1.0 + U * U / c->sigma_u2) * c->dsig2_dX;
}

int orc_normalise(orc_params* p) {
  if (!(p->u_star > 0.0) || !(p->kappa_sigma > 0.0) || !(p->kappa_tau > 0.0)) return -1;
  if (!(p->H > 0.0)) {
    if (!(p->f_coriolis > 0.0)) return -1;
    p->H = 0.3 * p->u_star / p->f_coriolis;
  }
  if (!(p->eps_reg_frac > 0.0) || !(p->eps_reg_frac <= 0.5)) return -1;
  if (!(p->T > 0.0) || p->M0 < 1 || p->level_min < 0) return -1;
  if (p->z_adapt < 0.0 || p->z_adapt > p->H) return -1;
  if (p->z_adapt > 0.0) {
    if (p->M0 > (1 << 22)) return -1;  /* T in ticks below 2^62 */
    /* lambda(X_adapt) >= lambda_max / 1024 bounds the steps per path */
    if (!(1024.0 * coefficients(p, p->z_adapt).lambda >= coefficients(p, 0.0).lambda)) return -1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Elastic reflection (Section 4, after Wilson and Flesch): while X is      */
/* outside [0, H] replace X by -X (bottom) or 2H - X (top) and U by -U; the */
/* parity S counts reflections at both walls (Section 4.1.1).  A state that */
/* leaves |X| <= 1e3 H or is not finite marks the path as diverged.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double X, U;
  int S;      /* (-1)^{n_refl} */
  int refl;   /* n_refl        */
  int bad;    /* diverged      */
} state_t;

static void reflect(const orc_params* p, state_t* s) {
  const double H = p->H;
  while (!s->bad && (s->X < 0.0 || s->X > H)) {
    if (!(fabs(s->X) <= 1e3 * H)) { s->bad = 1; break; }
    if (s->X < 0.0) s->X = -s->X; else s->X = 2.0 * H - s->X;
    s->U = -s->U;
    s->S = -s->S;
    s->refl += 1;
  }
  if (!isfinite(s->X) || !isfinite(s->U)) s->bad = 1;
}

/* ------------------------------------------------------------------------ */
/* Integrators.  Each step is split at the point where its normal enters:   */
/* pre() does the work before the noise and returns the coefficients the    */
/* O (or SE noise) term uses; post() applies the noise and finishes.  The   */
/* split lets the coupled driver read the parity S at the noise time.       */
/* ------------------------------------------------------------------------ */

/* Symplectic Euler, Eq. (MethodSymplecticEuler). */
static coef_t se_pre(const orc_params* p, state_t* s, double h) {
  (void)h;
  return coefficients(p, s->X);
}
static void se_post(const orc_params* p, state_t* s, double h, double xi, const coef_t* c) {
  double U1 = (1.0 - c->lambda * h) * s->U - dVdX(c, s->U) * h + c->sigma * sqrt(h) * xi;
  double X1 = s->X + U1 * h;
  s->U = U1; s->X = X1;
  reflect(p, s);
}

/* OU factor sigma * sqrt((1 - e^{-2 lambda h}) / (2 lambda)) of the O-step. */
static double ou_noise(const coef_t* c, double h) {
  double one_minus_e2 = -expm1(-2.0 * c->lambda * h); /* 1 - exp(-2 lambda h) */
  return c->sigma * sqrt(one_minus_e2 / (2.0 * c->lambda));
}

/* Geometric Langevin (OBA), Eq. (MethodSymplecticEulerOU): O-step with the
 * coefficients at X_n, B-step at (X_n, U*), A-step. */
static coef_t gl_pre(const orc_params* p, state_t* s, double h) {
  (void)h;
  return coefficients(p, s->X);
}
static void gl_post(const orc_params* p, state_t* s, double h, double xi, const coef_t* c) {
  double Ustar = exp(-c->lambda * h) * s->U + ou_noise(c, h) * xi;  /* O */
  double U1 = Ustar - dVdX(c, Ustar) * h;                              /* B */
  double X1 = s->X + U1 * h;                                           /* A */
  s->U = U1; s->X = X1;
  reflect(p, s);
}

/* BAOAB, Eq. (MethodBAOAB); the state is folded back into [0, H] after each
 * A half-step, so the O-step sees an in-domain X_{n+1/2}. */
static coef_t baoab_pre(const orc_params* p, state_t* s, double h) {
  coef_t cn = coefficients(p, s->X);
  double Uh = s->U - dVdX(&cn, s->U) * (h / 2.0);   /* B half-step */
  double Xh = s->X + Uh * (h / 2.0);                 /* A half-step */
  s->U = Uh; s->X = Xh;
  reflect(p, s);
  return coefficients(p, s->X);                      /* at X_{n+1/2} */
}
static void baoab_post(const orc_params* p, state_t* s, double h, double xi, const coef_t* c) {
  double Ustar = exp(-c->lambda * h) * s->U + ou_noise(c, h) * xi;  /* O */
  double X1 = s->X + Ustar * (h / 2.0);                                /* A half-step */
  s->U = Ustar; s->X = X1;
  reflect(p, s);
  coef_t c1 = coefficients(p, s->X);
  s->U = s->U - dVdX(&c1, s->U) * (h / 2.0);                           /* B half-step */
  if (!isfinite(s->U)) s->bad = 1;
}

static coef_t step_pre(int integ, const orc_params* p, state_t* s, double h) {
  if (integ == ORC_SE) return se_pre(p, s, h);
  if (integ == ORC_GL) return gl_pre(p, s, h);
  return baoab_pre(p, s, h);
}
static void step_post(int integ, const orc_params* p, state_t* s, double h, double xi,
                      const coef_t* c) {
  if (integ == ORC_SE) se_post(p, s, h, xi, c);
  else if (integ == ORC_GL) gl_post(p, s, h, xi, c);
  else baoab_post(p, s, h, xi, c);
}

/* ------------------------------------------------------------------------ */
/* Initial state.  w0_mode 0: (z0, w0) as given (the paper's fixed release, */
/* Section 6).  1: U0 ~ N(0, sigma_U(z0)^2).  2: the well-mixed state,      */
/* X0 ~ U(0, H) and U0 | X0 ~ N(0, sigma_U(X0)^2) (Section 2).  The random  */
/* draws use the reserved counter block 0xFFFFFFFF and are shared by the    */
/* fine and coarse path of a pair.                                          */
/* ------------------------------------------------------------------------ */
static void initial_state(const orc_params* p, int level, uint64_t i, uint64_t seed,
                          double* X0, double* U0) {
  *X0 = p->z0;
  *U0 = p->w0;
  if (p->w0_mode == 0) return;
  uint32_t x[4];
  philox_words(p, level, i, 0xFFFFFFFFu, seed, x);
  double xa, xb;
  box_muller(uniform01(p, x[0]), uniform01(p, x[1]), &xa, &xb);
  if (p->w0_mode == 2) *X0 = p->H * uniform01(p, x[2]);
  coef_t c = coefficients(p, *X0);
  *U0 = c.sigma_u * xa;
}

static void trace_put(double* tr, int row, const state_t* s) {
  if (!tr) return;
  tr[3 * row + 0] = s->X;
  tr[3 * row + 1] = s->U;
  tr[3 * row + 2] = (double)s->S;
}

static int steps_on_level(const orc_params* p, int level, int64_t* M) {
  if (level < 0 || level > 40) return -1;
  *M = (int64_t)p->M0 << level;
  return 0;
}

/* Normal xi_n of fine step n: element n mod 4 of the Philox block n / 4. */
typedef struct { uint32_t block; double xi[4]; } normal_cache_t;
static double normal_at(const orc_params* p, int level, uint64_t i, uint64_t seed,
                        normal_cache_t* nc, int64_t n) {
  uint32_t b = (uint32_t)(n / 4);
  if (b != nc->block) {
    orc_normals4(p, level, i, b, seed, nc->xi);
    nc->block = b;
  }
  return nc->xi[n % 4];
}

/* ------------------------------------------------------------------------ */
/* Adaptive, non-nested timesteps (Section 7.2, "Adaptive timestepping").     */
/*                                                                          */
/* Step rule, Eq. (adaptive h): h_n = min(h, lambda(X_adapt) / lambda(X_n) h) */
/* with X_n the path's own position at the start of its step (lambda of the */
/* regularised profile), and the last step of a path shortened to end at T. */
/* lambda decreases with height, so the ratio is below 1 exactly when the   */
/* clamped X_n lies below X_adapt; the step is then shortened to           */
/* floor(Q ratio) / Q of h, Q = 2^adapt_q (1024 by default; at least 1/1024 */
/* of h, which the parameter check guarantees): the same rule on every      */
/* level, never longer than the paper's step, and a decision that rounding  */
/* of lambda rarely flips.  With adapt_q = 30 it is the paper's rule to     */
/* 1e-9 relative.                                                           */
/* Time is counted in ticks of h_0 / 2^40 with h_0 = T / M0, so that h_l =  */
/* 2^(40 - l) ticks and every step is a whole number of ticks; the fine and */
/* coarse time points of a pair are compared exactly.                       */
/*                                                                          */
/* Coupling on the merged grid tau_0 = 0 < tau_1 < ... < T of the fine and  */
/* coarse time points: interval j carries the normal xi_j (element j mod 4  */
/* of Philox block j / 4, the counter the uniform path uses for fine step   */
/* j).  Over one step of a path the increments of the intervals inside it   */
/* combine as                                                               */
/*   SE, Eq. (AdaptivityIncrementEuler):                                    */
/*     dW = S_i^(c) sum_j S_j^(f) xi_j sqrt(tau_{j+1} - tau_j)               */
/*   GL, Eq. (AdaptivityIncrementSplitting):                                */
/*     A = S_i^(c) sum_j S_j^(f) xi_j sqrt((1 - e^{-2 lambda d_j}) / (2 lambda)) */
/*             exp(-lambda sum_{k > j} d_k),   d_j = tau_{j+1} - tau_j,       */
/* where dW replaces sqrt(h) xi in Eq. (MethodSymplecticEuler) and A        */
/* replaces sqrt((1 - e^{-2 lambda h}) / (2 lambda)) xi in the O-step of     */
/* Eq. (MethodSymplecticEulerOU).  For the fine path the parities are       */
/* dropped.  S_j^(f) is the fine parity at tau_j (fixed within a fine step),  */
/* S_i^(c) the coarse parity at the start of the coarse step.  lambda is the  */
/* stepping path's own lambda at the start of its step (the reading under   */
/* which A is exactly the OU noise integral over the step, so the coarse    */
/* path keeps the law of the fine path one level down).                     */
/* ------------------------------------------------------------------------ */
#define ORC_TICK_BITS 40

typedef struct {
  state_t s;
  coef_t c;        /* coefficients at the start of the current step */
  int64_t t_end;   /* tick at which the current step ends           */
  int64_t n;       /* ticks of the current step                     */
  double A;        /* noise accumulated over the step               */
  int64_t steps;
} astep_t;

/* Start a step at tick t: coefficients at X_n, the step rule, the cap at T. */
static void adapt_begin(const orc_params* p, astep_t* a, double lam_a, int64_t hmax,
                        int64_t t, int64_t T_ticks, double* tie) {
  a->c = coefficients(p, a->s.X);
  const double H = p->H, eps = p->eps_reg_frac * H;
  const double Xc = fmin(fmax(a->s.X, eps), H - eps);
  int64_t n = hmax;
  double m = fabs(Xc - p->z_adapt) / H;      /* margin of the "below X_adapt" test */
  if (Xc < p->z_adapt) {
    const int q = p->adapt_q > 0 ? p->adapt_q : 10;
    const double Q = ldexp(1.0, q);
    const double r = Q * (lam_a / a->c.lambda);
    double k = floor(r);
    const double mk = (r - k < k + 1.0 - r ? r - k : k + 1.0 - r) / Q;
    if (mk < m) m = mk;                        /* margin of the floor */
    if (k < 1.0) k = 1.0;
    if (k > Q) k = Q;
    n = (int64_t)k * (hmax >> q);
  }
  if (t > 0 && m < *tie) *tie = m;             /* the release point is exact on any side */
  if (n > T_ticks - t) n = T_ticks - t;
  a->n = n;
  a->t_end = t + n;
  a->A = 0.0;
}

/* Add the interval of d seconds with normal xi and parity weight w. */
static void adapt_accumulate(int integ, astep_t* a, double d, double xi, double w) {
  if (integ == ORC_SE) {
    a->A += w * sqrt(d) * xi;
  } else {
    const double lam = a->c.lambda;
    a->A = a->A * exp(-lam * d) + w * sqrt(-expm1(-2.0 * lam * d) / (2.0 * lam)) * xi;
  }
}

/* Finish the step with its accumulated noise times the parity factor Sx. */
static void adapt_step(const orc_params* p, int integ, astep_t* a, double h, double Sx) {
  state_t* s = &a->s;
  const coef_t* c = &a->c;
  if (integ == ORC_SE) {
    double U1 = (1.0 - c->lambda * h) * s->U - dVdX(c, s->U) * h + c->sigma * (Sx * a->A);
    s->U = U1;
    s->X = s->X + U1 * h;
  } else {
    double Ustar = exp(-c->lambda * h) * s->U + c->sigma * (Sx * a->A);  /* O */
    double U1 = Ustar - dVdX(c, Ustar) * h;                                /* B */
    s->U = U1;
    s->X = s->X + U1 * h;                                                  /* A */
  }
  reflect(p, s);
  a->steps += 1;
}

static int path_adaptive(const orc_params* p, int integ, int level, uint64_t i, uint64_t seed,
                         orc_path_out* out) {
  const int q = p->adapt_q > 0 ? p->adapt_q : 10;
  if (integ == ORC_BAOAB || q > 30 || level > ORC_TICK_BITS - q) return -1;
  const int coupled = level > p->level_min;
  const double lam_a = coefficients(p, p->z_adapt).lambda;
  const double h0 = p->T / (double)p->M0;
  const double sec = ldexp(h0, -ORC_TICK_BITS);           /* seconds per tick */
  const int64_t T_ticks = (int64_t)p->M0 << ORC_TICK_BITS;
  const int64_t hf = (int64_t)1 << (ORC_TICK_BITS - level);
  const int64_t hc = 2 * hf;
  double tie = 1.0, gap = 1.0;

  astep_t f, c;
  double X0, U0;
  initial_state(p, level, i, seed, &X0, &U0);
  memset(&f, 0, sizeof(f));
  f.s.X = X0; f.s.U = U0; f.s.S = 1;
  c = f;
  adapt_begin(p, &f, lam_a, hf, 0, T_ticks, &tie);
  if (coupled) adapt_begin(p, &c, lam_a, hc, 0, T_ticks, &tie);

  normal_cache_t nc;
  nc.block = 0xFFFFFFFFu;
  int64_t t = 0, j = 0;
  while (t < T_ticks && !(f.s.bad || (coupled && c.s.bad))) {
    int64_t t_next = f.t_end;
    if (coupled) {
      if (c.t_end < t_next) t_next = c.t_end;
      if (f.t_end != c.t_end) {
        const double m = (double)llabs(f.t_end - c.t_end) / (double)hf;
        if (m < gap) gap = m;
      }
    }
    const double d = (double)(t_next - t) * sec;
    const double xi = normal_at(p, level, i, seed, &nc, j);
    j += 1;
    const double Sf = (p->coupling == 1) ? 1.0 : (double)f.s.S;  /* S_j^(f) at tau_j */
    adapt_accumulate(integ, &f, d, xi, 1.0);
    if (coupled) adapt_accumulate(integ, &c, d, xi, Sf);
    t = t_next;
    if (t == f.t_end) {
      adapt_step(p, integ, &f, (double)f.n * sec, 1.0);
      if (t < T_ticks) adapt_begin(p, &f, lam_a, hf, t, T_ticks, &tie);
    }
    if (coupled && t == c.t_end) {
      const double Sc = (p->coupling == 1) ? 1.0 : (double)c.s.S;  /* S_i^(c) */
      adapt_step(p, integ, &c, (double)c.n * sec, Sc);
      if (t < T_ticks) adapt_begin(p, &c, lam_a, hc, t, T_ticks, &tie);
    }
  }
  out->zf = f.s.X; out->wf = f.s.U;
  out->zc = coupled ? c.s.X : 0.0;
  out->wc = coupled ? c.s.U : 0.0;
  out->nonfinite = (f.s.bad || (coupled && c.s.bad)) ? 1 : 0;
  out->refl_f = f.s.refl;
  out->refl_c = coupled ? c.s.refl : 0;
  out->pad_ = 0;
  out->steps_f = f.steps;
  out->steps_c = coupled ? c.steps : 0;
  out->tie = tie;
  out->gap = gap;
  return 0;
}

/* The uniform-timestep pair of orc_path; for BAOAB, half_f (3 * M doubles)
 * and half_c (3 * M/2) optionally receive (z, w, S) after the first half of
 * every step, i.e. after the fold that follows its first A half-step. */
static int path_pair(const orc_params* pin, int integ, int level, uint64_t i, uint64_t seed,
                     orc_path_out* out, double* trace_f, double* trace_c, double* half_f,
                     double* half_c) {
  orc_params pp = *pin;
  orc_params* p = &pp;
  if (orc_normalise(p) != 0) return -1;
  if (integ < ORC_SE || integ > ORC_BAOAB) return -1;
  if (level < p->level_min) return -1;
  int64_t M;
  if (steps_on_level(p, level, &M) != 0) return -1;
  const int coupled = level > p->level_min;
  if (coupled && (M % 2) != 0) return -1;
  if (p->z_adapt > 0.0) {
    if (trace_f || trace_c || half_f || half_c) return -1;
    return path_adaptive(p, integ, level, i, seed, out);
  }
  if ((half_f || half_c) && integ != ORC_BAOAB) return -1;
  const double h = p->T / (double)M;

  state_t f, c;
  double X0, U0;
  initial_state(p, level, i, seed, &X0, &U0);
  f.X = X0; f.U = U0; f.S = 1; f.refl = 0; f.bad = 0;
  c = f;
  trace_put(trace_f, 0, &f);
  if (coupled) trace_put(trace_c, 0, &c);

  normal_cache_t nc;
  nc.block = 0xFFFFFFFFu;
#define NORMAL(n) normal_at(p, level, i, seed, &nc, (n))

  if (!coupled) {
    /* plain Monte Carlo path on the coarsest level, Eq. (StMCestimator) */
    for (int64_t n = 0; n < M && !f.bad; ++n) {
      double xi = NORMAL(n);
      coef_t co = step_pre(integ, p, &f, h);
      trace_put(half_f, (int)n, &f);
      step_post(integ, p, &f, h, xi, &co);
      trace_put(trace_f, (int)(n + 1), &f);
    }
  } else {
    /* coupled fine/coarse pair driven by the same Brownian path (Section
     * 3.2), with the reflection-aware coarse increments of Eqs.
     * (euler_coupled_treatment) and (splitting_coupled_treatment). */
    for (int64_t k = 0; k < M / 2 && !(f.bad || c.bad); ++k) {
      double xa = NORMAL(2 * k);
      double xb = NORMAL(2 * k + 1);
      /* fine sub-step 2k */
      coef_t ca = step_pre(integ, p, &f, h);
      trace_put(half_f, (int)(2 * k), &f);
      int Sa = f.S;            /* S_n^{(f)} at the time xi_n is applied */
      step_post(integ, p, &f, h, xa, &ca);
      trace_put(trace_f, (int)(2 * k + 1), &f);
      /* fine sub-step 2k+1 */
      coef_t cb = step_pre(integ, p, &f, h);
      trace_put(half_f, (int)(2 * k + 1), &f);
      int Sb = f.S;            /* S_{n+1}^{(f)} */
      step_post(integ, p, &f, h, xb, &cb);
      trace_put(trace_f, (int)(2 * k + 2), &f);
      /* coarse step k with timestep 2h */
      coef_t cc = step_pre(integ, p, &c, 2.0 * h);
      trace_put(half_c, (int)k, &c);
      int Sc = c.S;            /* S_n^{(c)} */
      if (p->coupling == 1) { Sa = 1; Sb = 1; Sc = 1; }  /* naive coupling */
      double xc;
      if (integ == ORC_SE) {
        xc = (double)Sc / sqrt(2.0) * ((double)Sa * xa + (double)Sb * xb);
      } else {
        /* lambda(X_n) of the fine O-step of sub-step 2k */
        double e = exp(-ca.lambda * h);
        xc = (double)Sc * (e * (double)Sa * xa + (double)Sb * xb) / sqrt(e * e + 1.0);
      }
      step_post(integ, p, &c, 2.0 * h, xc, &cc);
      trace_put(trace_c, (int)(k + 1), &c);
    }
  }
#undef NORMAL
  out->zf = f.X; out->wf = f.U;
  out->zc = coupled ? c.X : 0.0;
  out->wc = coupled ? c.U : 0.0;
  out->nonfinite = (f.bad || (coupled && c.bad)) ? 1 : 0;
  out->refl_f = f.refl;
  out->refl_c = coupled ? c.refl : 0;
  out->pad_ = 0;
  out->steps_f = M;
  out->steps_c = coupled ? M / 2 : 0;
  out->tie = 1.0;
  out->gap = 1.0;
  return 0;
}

int orc_path(const orc_params* p, int integ, int level, uint64_t i, uint64_t seed,
             orc_path_out* out, double* trace_f, double* trace_c) {
  return path_pair(p, integ, level, i, seed, out, trace_f, trace_c, NULL, NULL);
}

int orc_path_half(const orc_params* p, int integ, int level, uint64_t i, uint64_t seed,
                  orc_path_out* out, double* half_f, double* half_c) {
  return path_pair(p, integ, level, i, seed, out, NULL, NULL, half_f, half_c);
}

/* ------------------------------------------------------------------------ */
/* Smoothed indicator, Section 5.1 (Eqs. conc, gr, SmoothedIndicator).      */
/* p_r(s) = sum_k c_k s^k, k = 0..r+1, solves                               */
/*   p(-1) = 1,  p(1) = 0,                                                  */
/*   int_{-1}^{1} s^j p(s) ds = (-1)^j / (j + 1),  j = 0..r-1,              */
/* with int_{-1}^{1} s^m ds = 2 / (m + 1) for even m and 0 for odd m.        */
/* Gaussian elimination with partial pivoting, FP64.                        */
/* ------------------------------------------------------------------------ */
int orc_smooth_poly(int r, double* coef) {
  if (r < 0 || r > 20) return -1;
  const int n = r + 2;
  double A[22][23];
  memset(A, 0, sizeof(A));
  for (int k = 0; k < n; ++k) {
    A[0][k] = (k % 2 == 0) ? 1.0 : -1.0;   /* p(-1) */
    A[1][k] = 1.0;                          /* p(1)  */
  }
  A[0][n] = 1.0;
  A[1][n] = 0.0;
  for (int j = 0; j < r; ++j) {
    for (int k = 0; k < n; ++k) {
      int m = j + k;
      A[2 + j][k] = (m % 2 == 0) ? 2.0 / (double)(m + 1) : 0.0;
    }
    A[2 + j][n] = ((j % 2 == 0) ? 1.0 : -1.0) / (double)(j + 1);
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
    if (A[piv][c] == 0.0) return -1;
    if (piv != c)
      for (int k = 0; k <= n; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
    for (int i = c + 1; i < n; ++i) {
      double f = A[i][c] / A[c][c];
      for (int k = c; k <= n; ++k) A[i][k] -= f * A[c][k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = A[i][n];
    for (int k = i + 1; k < n; ++k) v -= A[i][k] * coef[k];
    coef[i] = v / A[i][i];
  }
  return 0;
}

double orc_g(int r, const double* coef, double x) {
  if (x < -1.0) return 1.0;
  if (x > 1.0) return 0.0;
  double v = 0.0;
  for (int k = r + 1; k >= 0; --k) v = v * x + coef[k];
  return v;
}

/* P^{r,delta}_{[a,b]}(X) = g_r((X - b) / delta) - g_r((X - a) / delta). */
static double smoothed_interval(const orc_params* p, const double* coef, double X) {
  return orc_g(p->smooth_r, coef, (X - p->qoi_b) / p->smooth_delta) -
         orc_g(p->smooth_r, coef, (X - p->qoi_a) / p->smooth_delta);
}

/* ------------------------------------------------------------------------ */
/* Level sums, Eq. (Yhatell): Y = P_l - P_{l-1} per pair (Y = P on the      */
/* coarsest level), for the QoIs P = X_T and P = 1[X_T < threshold].  Sums  */
/* use Neumaier's compensated summation in a fixed order: paths in chunks   */
/* of CHUNK, chunks combined in index order, whatever the thread count.     */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } csum_t;
static void csum_add(csum_t* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double csum_val(const csum_t* a) { return a->s + a->c; }

#define CHUNK 1024u
typedef struct {
  csum_t sum[2][6];
  uint64_t n, bad, steps;
} chunk_t;

typedef struct {
  const orc_params* p;
  const double* coef;       /* smoothing polynomial when qoi1_mode == 1 */
  int integ, level;
  uint64_t offset, N, seed;
  uint64_t first_chunk, n_chunks;
  chunk_t* chunks;
  volatile uint64_t* next;  /* shared chunk counter */
  pthread_mutex_t* lock;
} work_t;

static void run_chunk(const work_t* w, uint64_t chunk, chunk_t* out) {
  memset(out, 0, sizeof(*out));
  const int coupled = w->level > w->p->level_min;
  uint64_t a = chunk * CHUNK, b = a + CHUNK;
  if (b > w->N) b = w->N;
  for (uint64_t j = a; j < b; ++j) {
    orc_path_out r;
    orc_path(w->p, w->integ, w->level, w->offset + j, w->seed, &r, NULL, NULL);
    out->steps += (uint64_t)(r.steps_f + r.steps_c);
    if (r.nonfinite) { out->bad++; continue; }
    double Pf[2], Pc[2];
    Pf[0] = r.zf;
    Pc[0] = coupled ? r.zc : 0.0;
    if (w->p->qoi1_mode == 1) {
      Pf[1] = smoothed_interval(w->p, w->coef, r.zf);
      Pc[1] = coupled ? smoothed_interval(w->p, w->coef, r.zc) : 0.0;
    } else {
      Pf[1] = (r.zf < w->p->qoi_threshold) ? 1.0 : 0.0;
      Pc[1] = coupled ? ((r.zc < w->p->qoi_threshold) ? 1.0 : 0.0) : 0.0;
    }
    for (int q = 0; q < 2; ++q) {
      double Y = Pf[q] - Pc[q];
      csum_add(&out->sum[q][0], Y);
      csum_add(&out->sum[q][1], Y * Y);
      csum_add(&out->sum[q][2], Pf[q]);
      csum_add(&out->sum[q][3], Pf[q] * Pf[q]);
      csum_add(&out->sum[q][4], Pc[q]);
      csum_add(&out->sum[q][5], Pc[q] * Pc[q]);
    }
    out->n++;
  }
}

static void* worker(void* arg) {
  work_t* w = (work_t*)arg;
  for (;;) {
    uint64_t k;
    pthread_mutex_lock(w->lock);
    k = *w->next;
    *w->next = k + 1;
    pthread_mutex_unlock(w->lock);
    if (k >= w->n_chunks) break;
    run_chunk(w, w->first_chunk + k, &w->chunks[k]);
  }
  return NULL;
}

int orc_level_sums(const orc_params* pin, int integ, int level, uint64_t N,
                   uint64_t offset, uint64_t seed, int threads, orc_level_sums_t* out) {
  orc_params pp = *pin;
  if (orc_normalise(&pp) != 0) return -1;
  if (integ < ORC_SE || integ > ORC_BAOAB || level < pp.level_min) return -1;
  int64_t M;
  if (steps_on_level(&pp, level, &M) != 0) return -1;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  double coef[24];
  if (pp.qoi1_mode == 1 && (orc_smooth_poly(pp.smooth_r, coef) != 0 || !(pp.smooth_delta > 0.0)))
    return -1;

  csum_t tot[2][6];
  memset(tot, 0, sizeof(tot));
  uint64_t n_ok = 0, n_bad = 0, n_steps = 0;
  const uint64_t n_chunks_all = (N + CHUNK - 1) / CHUNK;
  const uint64_t BATCH = 4096; /* chunks per batch, bounds memory */
  chunk_t* chunks = (chunk_t*)malloc(sizeof(chunk_t) * BATCH);
  if (!chunks) return -1;
  pthread_mutex_t lock;
  pthread_mutex_init(&lock, NULL);
  for (uint64_t first = 0; first < n_chunks_all; first += BATCH) {
    uint64_t nb = n_chunks_all - first;
    if (nb > BATCH) nb = BATCH;
    volatile uint64_t next = 0;
    work_t w;
    w.p = &pp; w.coef = coef; w.integ = integ; w.level = level; w.offset = offset; w.N = N;
    w.seed = seed; w.first_chunk = first; w.n_chunks = nb; w.chunks = chunks;
    w.next = &next; w.lock = &lock;
    int nt = threads;
    if ((uint64_t)nt > nb) nt = (int)nb;
    if (nt <= 1) {
      worker(&w);
    } else {
      pthread_t tid[256];
      for (int t = 0; t < nt; ++t) pthread_create(&tid[t], NULL, worker, &w);
      for (int t = 0; t < nt; ++t) pthread_join(tid[t], NULL);
    }
    for (uint64_t k = 0; k < nb; ++k) {
      for (int q = 0; q < 2; ++q)
        for (int j = 0; j < 6; ++j) csum_add(&tot[q][j], csum_val(&chunks[k].sum[q][j]));
      n_ok += chunks[k].n;
      n_bad += chunks[k].bad;
      n_steps += chunks[k].steps;
    }
  }
  pthread_mutex_destroy(&lock);
  free(chunks);
  memset(out, 0, sizeof(*out));
  out->n = n_ok;
  out->n_nonfinite = n_bad;
  /* integrator steps executed, fine + coarse (M + M/2 per pair with
   * uniform timesteps) */
  out->path_steps = n_steps;
  for (int q = 0; q < 2; ++q)
    for (int j = 0; j < 6; ++j) out->sum[q][j] = csum_val(&tot[q][j]);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Adaptive MLMC driver: the algorithm of Giles (2008, Operations Research, */
/* Section 5) that the paper uses to pick N_l on the fly (Section 6, second */
/* paragraph):                                                              */
/*   1. start with L = level_min                                            */
/*   2. estimate V_L with n_init samples                                    */
/*   3. optimal N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k))    */
/*      (Giles 2008 Eq. 12, with C_l the path-steps of one sample)          */
/*   4. evaluate the extra samples each level needs                         */
/*   5. if L >= level_min + 2, converged when                               */
/*      max(|Yhat_{L-1}| / 2, |Yhat_L|) < eps / sqrt(2)  (Giles Eq. 11, M=2) */
/*   6. otherwise L := L + 1 (up to L_max) and go to 2.                     */
/* N_l is driven by QoI 0 (the mean position).                              */
/* ------------------------------------------------------------------------ */
static void merge_sums(orc_level_sums_t* a, const orc_level_sums_t* b) {
  a->n += b->n;
  a->n_nonfinite += b->n_nonfinite;
  a->path_steps += b->path_steps;
  for (int q = 0; q < 2; ++q)
    for (int j = 0; j < 6; ++j) a->sum[q][j] += b->sum[q][j];
}

int orc_estimate(const orc_params* pin, int integ, double eps, uint64_t seed,
                 int threads, orc_result_t* out) {
  orc_params pp = *pin;
  orc_params* p = &pp;
  if (orc_normalise(p) != 0 || !(eps > 0.0)) return -1;
  if (p->L_max < p->level_min + 2 || p->L_max >= ORC_MAX_LEVELS) return -1;
  if (p->n_init < 2) return -1;
  orc_level_sums_t S[ORC_MAX_LEVELS];
  uint64_t Ndone[ORC_MAX_LEVELS], dN[ORC_MAX_LEVELS];
  double V[ORC_MAX_LEVELS], C[ORC_MAX_LEVELS];
  memset(S, 0, sizeof(S));
  memset(Ndone, 0, sizeof(Ndone));
  memset(dN, 0, sizeof(dN));
  const int lmin = p->level_min;
  int L = lmin;
  int converged = 0;
  for (;;) {
    dN[L] = (uint64_t)p->n_init;                             /* step 2 */
    for (int pass = 0; pass < 2; ++pass) {
      /* pass 0 runs the n_init samples of the new level; pass 1 (steps 3 and
       * 4) runs the extra samples the updated N_l ask for. */
      for (int l = lmin; l <= L; ++l) {
        if (dN[l] == 0) continue;
        orc_level_sums_t r;
        if (orc_level_sums(p, integ, l, dN[l], Ndone[l], seed, threads, &r) != 0) return -1;
        merge_sums(&S[l], &r);
        Ndone[l] += dN[l];
        dN[l] = 0;
      }
      if (pass == 1) break;
      double total = 0.0;                                      /* step 3 */
      for (int l = lmin; l <= L; ++l) {
        double n = (double)S[l].n;
        double m1 = S[l].sum[0][0], m2 = S[l].sum[0][1];
        V[l] = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
        if (V[l] < 0.0) V[l] = 0.0;
        /* C_l: integrator steps of one sample (measured: fixed with uniform
         * timesteps, state-dependent with adaptive ones) */
        C[l] = (double)S[l].path_steps / (double)(S[l].n + S[l].n_nonfinite);
        total += sqrt(V[l] * C[l]);
      }
      for (int l = lmin; l <= L; ++l) {
        double Nopt = ceil(2.0 / (eps * eps) * sqrt(V[l] / C[l]) * total);
        dN[l] = (Nopt > (double)Ndone[l]) ? (uint64_t)(Nopt - (double)Ndone[l]) : 0;
      }
    }
    if (L >= lmin + 2) {                                       /* step 5 */
      double yL = fabs(S[L].sum[0][0] / (double)S[L].n);
      double yL1 = fabs(S[L - 1].sum[0][0] / (double)S[L - 1].n);
      double rem = fmax(yL1 / 2.0, yL);
      if (rem < eps / sqrt(2.0)) { converged = 1; break; }
    }
    if (L >= p->L_max) break;
    L += 1;                                                    /* step 6 */
  }
  memset(out, 0, sizeof(*out));
  out->L = L;
  out->converged = converged;
  for (int q = 0; q < 2; ++q) {
    double est = 0.0, var = 0.0;
    for (int l = lmin; l <= L; ++l) {
      double n = (double)S[l].n;
      double m1 = S[l].sum[q][0], m2 = S[l].sum[q][1];
      est += m1 / n;
      double v = n > 1.0 ? (m2 - m1 * m1 / n) / (n - 1.0) : 0.0;
      var += (v > 0.0 ? v : 0.0) / n;
    }
    out->estimate[q] = est;
    out->est_variance[q] = var;
  }
  for (int l = lmin; l <= L; ++l) {
    out->N[l] = S[l].n;
    double n = (double)S[l].n;
    out->mean_y[l] = S[l].sum[0][0] / n;
    double v = n > 1.0 ? (S[l].sum[0][1] - S[l].sum[0][0] * S[l].sum[0][0] / n) / (n - 1.0) : 0.0;
    out->V[l] = v > 0.0 ? v : 0.0;
    out->total_path_steps += S[l].path_steps;
    out->n_nonfinite += S[l].n_nonfinite;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Binned density, Section 6.3 (Eq. vector_QoI): bin i = [a_i, a_{i+1}),    */
/* a_i = i H / k, QoI P_i = P^{r,delta}_{[a_i, a_{i+1}]}(X_T); per bin the   */
/* six sums of Y_i = P_i(fine) - P_i(coarse).  Same fixed chunk order and    */
/* Neumaier sums as orc_level_sums.                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_params* p;
  const double* coef;
  int integ, level, k;
  uint64_t offset, N, seed, n_chunks;
  csum_t* sums;        /* n_chunks x k x 6 */
  uint64_t* n_ok;      /* n_chunks */
  volatile uint64_t* next;
  pthread_mutex_t* lock;
} pdf_work_t;

static void pdf_chunk(const pdf_work_t* w, uint64_t chunk) {
  const orc_params* p = w->p;
  const int coupled = w->level > p->level_min;
  const int k = w->k;
  csum_t* S = w->sums + chunk * (uint64_t)k * 6;
  memset(S, 0, sizeof(csum_t) * (size_t)k * 6);
  w->n_ok[chunk] = 0;
  uint64_t a = chunk * CHUNK, b = a + CHUNK;
  if (b > w->N) b = w->N;
  for (uint64_t j = a; j < b; ++j) {
    orc_path_out r;
    orc_path(p, w->integ, w->level, w->offset + j, w->seed, &r, NULL, NULL);
    if (r.nonfinite) continue;
    for (int i = 0; i < k; ++i) {
      double lo = p->H * (double)i / (double)k, hi = p->H * (double)(i + 1) / (double)k;
      double Pf = orc_g(p->smooth_r, w->coef, (r.zf - hi) / p->smooth_delta) -
                  orc_g(p->smooth_r, w->coef, (r.zf - lo) / p->smooth_delta);
      double Pc = 0.0;
      if (coupled)
        Pc = orc_g(p->smooth_r, w->coef, (r.zc - hi) / p->smooth_delta) -
             orc_g(p->smooth_r, w->coef, (r.zc - lo) / p->smooth_delta);
      double Y = Pf - Pc;
      csum_add(&S[6 * i + 0], Y);
      csum_add(&S[6 * i + 1], Y * Y);
      csum_add(&S[6 * i + 2], Pf);
      csum_add(&S[6 * i + 3], Pf * Pf);
      csum_add(&S[6 * i + 4], Pc);
      csum_add(&S[6 * i + 5], Pc * Pc);
    }
    w->n_ok[chunk] += 1;
  }
}

static void* pdf_worker(void* arg) {
  pdf_work_t* w = (pdf_work_t*)arg;
  for (;;) {
    uint64_t c;
    pthread_mutex_lock(w->lock);
    c = *w->next;
    *w->next = c + 1;
    pthread_mutex_unlock(w->lock);
    if (c >= w->n_chunks) break;
    pdf_chunk(w, c);
  }
  return NULL;
}

int orc_level_pdf_sums(const orc_params* pin, int integ, int level, uint64_t N, uint64_t offset,
                       uint64_t seed, int k, int threads, uint64_t* n_ok, double* out) {
  orc_params pp = *pin;
  if (orc_normalise(&pp) != 0) return -1;
  if (integ < ORC_SE || integ > ORC_BAOAB || level < pp.level_min || k < 1 || k > 256) return -1;
  if (!(pp.smooth_delta > 0.0)) return -1;
  double coef[24];
  if (orc_smooth_poly(pp.smooth_r, coef) != 0) return -1;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  const uint64_t n_chunks = (N + CHUNK - 1) / CHUNK;
  csum_t* sums = (csum_t*)malloc(sizeof(csum_t) * (size_t)(n_chunks ? n_chunks : 1) * k * 6);
  uint64_t* nk = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n_chunks ? n_chunks : 1));
  if (!sums || !nk) { free(sums); free(nk); return -1; }
  pthread_mutex_t lock;
  pthread_mutex_init(&lock, NULL);
  volatile uint64_t next = 0;
  pdf_work_t w;
  w.p = &pp; w.coef = coef; w.integ = integ; w.level = level; w.k = k;
  w.offset = offset; w.N = N; w.seed = seed; w.n_chunks = n_chunks;
  w.sums = sums; w.n_ok = nk; w.next = &next; w.lock = &lock;
  int nt = threads;
  if ((uint64_t)nt > n_chunks) nt = (int)(n_chunks ? n_chunks : 1);
  if (nt <= 1) {
    pdf_worker(&w);
  } else {
    pthread_t tid[256];
    for (int t = 0; t < nt; ++t) pthread_create(&tid[t], NULL, pdf_worker, &w);
    for (int t = 0; t < nt; ++t) pthread_join(tid[t], NULL);
  }
  pthread_mutex_destroy(&lock);
  uint64_t tot_n = 0;
  for (int i = 0; i < k * 6; ++i) {
    csum_t acc = {0.0, 0.0};
    for (uint64_t c = 0; c < n_chunks; ++c) csum_add(&acc, csum_val(&sums[c * (uint64_t)k * 6 + i]));
    out[i] = csum_val(&acc);
  }
  for (uint64_t c = 0; c < n_chunks; ++c) tot_n += nk[c];
  *n_ok = tot_n;
  free(sums);
  free(nk);
  return 0;
}
