/*
 * oracle.h -- plain, slow FP64 CPU oracle for the MLMC boundary-layer
 * dispersion path of Katsiolides, Mueller, Scheichl, Shardlow, Giles and
 * Thomson, "Multilevel Monte Carlo and improved timestepping methods in
 * atmospheric dispersion modelling" (arXiv 1612.07717).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) includes, links or calls this code; only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark do.  It shares no
 * code, header, table or constant with the CUDA path: the Philox generator
 * and the normal map are implemented here a second time from their published
 * definitions.
 *
 * Every quantity is double precision.  Each function names the passage of
 * the paper it restates.
 */
#ifndef MLMC_ORACLE_H
#define MLMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SE = 0, ORC_GL = 1, ORC_BAOAB = 2 };
/* uniform map applied to one 32-bit Philox word */
enum { ORC_U23 = 0,   /* u = (floor(x / 2^9) + 1/2) * 2^-23 : the FP32 kernel's map */
       ORC_U32 = 1 }; /* u = (x + 1/2) * 2^-32                : the FP64 kernel's map */

typedef struct {
  double u_star;        /* friction velocity u* [m/s]                              */
  double f_coriolis;    /* Coriolis parameter f [1/s]                              */
  double H;             /* boundary-layer depth [m]; <= 0 means 0.3 u* / f           */
  double kappa_sigma;   /* 1.3  (Eq. profiles)                                     */
  double kappa_tau;     /* 0.5  (Eq. profiles)                                     */
  double c_f;           /* tau divided by (1 + c_f f z / u*); 0 gives the paper's tau */
  double eps_reg_frac;  /* regularisation height eps_reg as a fraction of H        */
  double z0, w0;        /* release height [m], fixed release velocity [m/s]        */
  double T;             /* travel time [s]                                         */
  double qoi_threshold; /* indicator QoI: 1[z(T) < qoi_threshold] [m]              */
  int32_t w0_mode;      /* 0 fixed w0; 1 w0 ~ N(0, sigma_w(z0)^2); 2 well mixed    */
  int32_t M0;           /* timesteps on level 0; level l uses M0 * 2^l             */
  int32_t level_min;    /* coarsest level of the hierarchy (plain MC on it)         */
  int32_t L_max;        /* finest level the adaptive driver may add                 */
  int32_t coupling;     /* 0 reflection-aware coupling; 1 naive (all S = 1)         */
  int32_t drift_outside;/* 0 d(sigma_w^2)/dz = 0 outside the band; 1 frozen value   */
  int32_t n_init;       /* initial samples on a new level (adaptive driver)         */
  int32_t uniform_map;  /* ORC_U23 or ORC_U32                                       */
  uint32_t stream_id;   /* Philox counter word 3 (one stream per query)             */
  int32_t qoi1_mode;    /* QoI 1: 0 indicator 1[z(T) < qoi_threshold];
                           1 smoothed interval P^{r,delta}_{[qoi_a, qoi_b]}(z(T))     */
  double qoi_a, qoi_b;  /* interval of the smoothed QoI [m]                          */
  double smooth_delta;  /* smoothing width delta [m]                                 */
  int32_t smooth_r;     /* smoothing order r (p_r has degree r + 1)                  */
  int32_t adapt_q;      /* adaptive timesteps: a shortened step is a whole number
                           of 2^-adapt_q of h; 0 means 10 (the CUDA library's
                           1/1024); up to 30, where the rule is the paper's
                           min(h, lambda(X_adapt) / lambda(X_n) h) to 1e-9
                           relative (needs level <= 40 - adapt_q)              */
  double z_adapt;       /* > 0: adaptive timesteps with reference height X_adapt [m]
                           (Section 7.2, SE and GL only; needs z_adapt <= H,
                           M0 <= 2^22 and lambda(X_adapt) >= lambda_max / 1024);
                           0: uniform timesteps                                 */
} orc_params;

typedef struct {
  double zf, wf, zc, wc; /* final states of the fine and coarse path          */
  int32_t nonfinite;     /* 1 if either path left |z| <= 1e3 H or became NaN  */
  int32_t refl_f, refl_c;/* number of reflections on each path                */
  int32_t pad_;
  int64_t steps_f, steps_c; /* integrator steps taken by each path             */
  double tie;            /* adaptive timesteps: smallest margin of a step
                            decision (see orc_path); 1 for uniform timesteps */
  double gap;            /* adaptive timesteps: smallest |t_f - t_c| / h over
                            distinct next fine and coarse time points; 1 for
                            uniform timesteps                                */
} orc_path_out;

/* per QoI q (0: z(T), 1: 1[z(T) < threshold]) the six sums
 * sum[q] = { sum Y, sum Y^2, sum P_f, sum P_f^2, sum P_c, sum P_c^2 } */
typedef struct {
  uint64_t n;           /* finite paths that entered the sums  */
  uint64_t path_steps;  /* integrator steps executed (fine + coarse) */
  uint64_t n_nonfinite; /* paths excluded as diverged          */
  uint64_t pad_;
  double sum[2][6];
} orc_level_sums_t;

#define ORC_MAX_LEVELS 32
typedef struct {
  double estimate[2];        /* MLMC estimate of E[P] per QoI                  */
  double est_variance[2];    /* sum_l V_l / N_l per QoI                          */
  int32_t L;                 /* finest level used                                */
  int32_t converged;         /* 1 if the bias test passed before L_max           */
  uint64_t N[ORC_MAX_LEVELS];     /* samples per level (index = level)           */
  double V[ORC_MAX_LEVELS];       /* sample variance of Y_l (QoI 0)              */
  double mean_y[ORC_MAX_LEVELS];  /* mean of Y_l (QoI 0)                         */
  uint64_t total_path_steps;
  uint64_t n_nonfinite;
} orc_result_t;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The four standard normals of fine steps 4k..4k+3 of path i on level l. */
void orc_normals4(const orc_params* p, int level, uint64_t i, uint32_t block,
                  uint64_t seed, double xi[4]);

/* sigma_w, sigma_w^2, d(sigma_w^2)/dz, lambda, sigma at height z. */
void orc_coefficients(const orc_params* p, double z, double out[5]);

/* Fill defaults that depend on others (H from u*, f).  Returns 0 or -1. */
int orc_normalise(orc_params* p);

/* One coupled path pair of level `level` (fine only when level ==
 * level_min).  trace_f (3 * (M+1) doubles: z, w, S per fine time point) and
 * trace_c (3 * (M/2+1)) are optional (uniform timesteps only).  With
 * p->z_adapt > 0 the pair takes the adaptive, non-nested timesteps of
 * Section 7.2 on the merged time grid; time is counted in ticks of
 * h_0 / 2^40 (h_0 = T / M0) and each adaptive step is a whole number of
 * ticks; a shortened step is floor(Q lambda(X_adapt) / lambda(X_n)) / Q of h,
 * Q = 2^adapt_q (1024 by default).  out->tie is the smallest margin of a
 * step decision after the release: |X_n - X_adapt| / H for "below X_adapt",
 * and the distance of Q lambda(X_adapt) / lambda(X_n) to an integer, over Q,
 * for the floor.  Where it is tiny, a rounding difference can change a step and with
 * it the merged grid.  out->gap is the smallest |t_f - t_c| / h over distinct next
 * fine and coarse time points (a rounding difference there only moves a
 * short interval between neighbouring steps).  Returns 0, or -1 on bad
 * arguments. */
int orc_path(const orc_params* p, int integ, int level, uint64_t i, uint64_t seed,
             orc_path_out* out, double* trace_f, double* trace_c);

/* orc_path for BAOAB with uniform timesteps, recording (z, w, S) after the
 * first half of every step -- the state after the fold that follows the
 * first A half-step (Eq. MethodBAOAB), where the noise of the step enters --
 * into half_f (3 * M doubles, row n for fine step n) and, on coupled levels,
 * half_c (3 * M/2 doubles); either may be NULL.  Returns -1 for another
 * integrator, adaptive timesteps or bad arguments. */
int orc_path_half(const orc_params* p, int integ, int level, uint64_t i, uint64_t seed,
                  orc_path_out* out, double* half_f, double* half_c);

/* Level sums over paths [offset, offset + N).  threads <= 0 uses 1.  The
 * result does not depend on the thread count. */
int orc_level_sums(const orc_params* p, int integ, int level, uint64_t N,
                   uint64_t offset, uint64_t seed, int threads, orc_level_sums_t* out);

/* Smoothing polynomial p_r of Section 5.1: degree r + 1, p(-1) = 1,
 * p(1) = 0, and its first r moments on [-1, 1] equal those of the step
 * function.  coef[k] multiplies s^k, k = 0..r+1.  Returns 0 or -1. */
int orc_smooth_poly(int r, double* coef);

/* g_r(x): 1 for x < -1, p_r(x) on [-1, 1], 0 for x > 1 (Eq. gr). */
double orc_g(int r, const double* coef, double x);

/* Level sums of the binned density (Section 6.3, Eq. vector_QoI): k bins
 * [i H / k, (i + 1) H / k), each QoI the smoothed interval P^{r,delta};
 * out[6 * i + j] as the six sums of orc_level_sums for bin i. */
int orc_level_pdf_sums(const orc_params* p, int integ, int level, uint64_t N, uint64_t offset,
                       uint64_t seed, int k, int threads, uint64_t* n_ok, double* out);

/* Adaptive MLMC estimate of E[z(T)] to RMSE eps (Giles 2008, Section 5). */
int orc_estimate(const orc_params* p, int integ, double eps, uint64_t seed,
                 int threads, orc_result_t* out);

#ifdef __cplusplus
}
#endif
#endif
