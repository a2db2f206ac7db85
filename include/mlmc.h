/*
 * mlmc.h -- C ABI of the GB300 (sm_103a) library for multilevel Monte Carlo
 * estimation of particle dispersion in a 1-D atmospheric boundary layer, after
 * Katsiolides, Mueller, Scheichl, Shardlow, Giles and Thomson, "Multilevel
 * Monte Carlo and improved timestepping methods in atmospheric dispersion
 * modelling" (arXiv 1612.07717).
 *
 * The problem (Section 2, Eq. generalised): a particle at height z with
 * vertical velocity w follows
 *     dw = [-w / tau(z) + 1/2 (1 + w^2 / sigma_w^2) d sigma_w^2/dz] dt
 *          + sqrt(2 sigma_w^2 / tau) dW,        dz = w dt,
 * reflected elastically at z = 0 and z = H (Section 4).  The library
 * estimates E[phi(z(T))] for phi(z) = z and phi(z) = 1[z < threshold] with
 * plain Monte Carlo (Eq. StMCestimator) or multilevel Monte Carlo (Eqs.
 * telescoping_sum, mlmcestimator, Yhatell), using the symplectic Euler,
 * geometric Langevin or BAOAB integrator (Section 3.1) and the
 * reflection-aware coupling of fine and coarse paths (Eqs.
 * euler_coupled_treatment and splitting_coupled_treatment).
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers; all others are host pointers.
 *  - The caller owns all memory.  The library never allocates device memory:
 *    device scratch is the caller's `workspace` of `ws_bytes` bytes, sized by
 *    mlmc_workspace_bytes().  Host output structs are written in place.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Kernels are
 *    launched on it.  Entry points that return results in a host struct
 *    synchronise that stream before returning; *_async entry points do not.
 *  - Return value: MLMC_OK (0) or a negative mlmc_status.  On an error no
 *    output is valid unless stated.  mlmc_strerror() names the code.
 *  - Random numbers: Philox4x32-10 with key = seed and counter =
 *    (step_block, path_lo, path_hi ^ (level << 24), stream_id); fine step n
 *    of a path (with adaptive timesteps: merged interval n of the pair)
 *    uses word n mod 4 of block n / 4, Box-Muller on word pairs.
 *    A path's samples therefore depend only on (seed, stream_id, level, path
 *    index): splitting [0, N) into calls over [0, a) and [a, N) with
 *    path_offset gives the same paths.
 */
#ifndef MLMC_GB300_H
#define MLMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
typedef enum {
  MLMC_OK = 0,
  MLMC_EINVAL = -1,      /* invalid argument or parameter                      */
  MLMC_EWORKSPACE = -2,  /* workspace NULL, misaligned or too small             */
  MLMC_ECUDA = -3,       /* a CUDA call failed (launch, copy, sync)             */
  MLMC_ENONFINITE = -4,  /* some paths diverged; they are excluded and counted,
                            every other output is valid                        */
  MLMC_ETIMEOUT = -5,    /* a device-side work loop hit its iteration limit    */
  MLMC_EUNSTABLE = -6,   /* symplectic Euler requested with h lambda_max >= 2   */
  MLMC_ENOTCONV = -7,    /* adaptive driver reached L_max before its bias test
                            passed; the estimate is still returned              */
  MLMC_ENODEV = -8,      /* no CUDA device or unsupported architecture          */
  MLMC_ECOMM = -9        /* the all-reduce hook failed, or another rank of a
                            sharded estimate reported an error                  */
} mlmc_status;

typedef enum { MLMC_SE = 0, MLMC_GL = 1, MLMC_BAOAB = 2 } mlmc_integrator;
typedef enum { MLMC_FP32 = 0, MLMC_FP64 = 1 } mlmc_precision;

/* ------------------------------------------------------------- parameters */
/* Scenario and hierarchy.  Profiles (Eq. profiles, Eq. regularisation):
 *   z_c     = clamp(z, eps_reg, H - eps_reg),  eps_reg = eps_reg_frac * H
 *   sigma_w = kappa_sigma u* (1 - z_c / H)^(3/4)
 *   tau     = kappa_tau z_c / sigma_w / (1 + c_f f z_c / u*)
 *   d sigma_w^2 / dz of the regularised profile (0 outside the band).
 * Level l integrates M0 * 2^l steps of h = T / (M0 2^l); the coarsest level
 * level_min is plain Monte Carlo, finer levels are coupled pairs. */
typedef struct mlmc_params {
  double u_star;        /* friction velocity u* [m/s], > 0                    */
  double f_coriolis;    /* Coriolis parameter f [1/s], >= 0                    */
  double H;             /* boundary-layer depth [m]; <= 0 selects 0.3 u* / f   */
  double kappa_sigma;   /* 1.3                                                  */
  double kappa_tau;     /* 0.5                                                  */
  double c_f;           /* Coriolis factor on tau (15; 0 = the paper's tau)     */
  double eps_reg_frac;  /* eps_reg / H, in (0, 0.5]                             */
  double z0;            /* release height [m] (w0_mode 0 and 1)                 */
  double w0;            /* release velocity [m/s] (w0_mode 0)                   */
  double T;             /* travel time [s], > 0                                 */
  double qoi_threshold; /* indicator QoI 1[z(T) < qoi_threshold] [m]            */
  int32_t w0_mode;      /* 0 fixed (z0, w0); 1 w0 ~ N(0, sigma_w(z0)^2);
                           2 well mixed z0 ~ U(0, H), w0 ~ N(0, sigma_w(z0)^2)  */
  int32_t M0;           /* steps on level 0, >= 1                                */
  int32_t level_min;    /* coarsest level (plain Monte Carlo on it)              */
  int32_t L_max;        /* finest level the adaptive driver may use, < 32        */
  int32_t coupling;     /* 0 reflection-aware (paper); 1 naive S = 1 (for study) */
  int32_t drift_outside;/* 0 d sigma_w^2/dz = 0 outside the band; 1 frozen value */
  int32_t n_init;       /* samples on a newly added level (adaptive driver)      */
  int32_t precision;    /* mlmc_precision of the path arithmetic                 */
  uint32_t stream_id;   /* Philox counter word 3: one random stream per query    */
  int32_t allow_unstable; /* 1: run SE levels with h lambda_max >= 2 anyway      */
  int32_t qoi1_mode;    /* QoI 1: 0 indicator 1[z(T) < qoi_threshold]; 1 smoothed
                           interval P^{r,delta}_{[qoi_a, qoi_b]}(z(T)) of Section 5.1
                           (Eq. SmoothedIndicator)                                */
  int32_t smooth_r;     /* smoothing order r, 0..10 (p_r has degree r + 1)      */
  double qoi_a, qoi_b;  /* interval of the smoothed QoI [m], qoi_a < qoi_b       */
  double smooth_delta;  /* smoothing width delta [m], > 0 when smoothing is used */
  double z_adapt;       /* 0: uniform timesteps.  > 0: adaptive, non-nested
                           timesteps with reference height X_adapt = z_adapt [m]
                           (Section 7.2): below X_adapt a step is shortened to
                           floor(1024 lambda(X_adapt) / lambda(X_n)) / 1024 of h
                           (the paper's min(h, lambda(X_adapt) / lambda(X_n) h)
                           rounded down to a 1024th of h), the coupled pair is
                           driven on the merged time grid.  SE and GL only;
                           needs 0 < z_adapt <= H, M_l <= 2^20 on the levels
                           used, and lambda(X_adapt) >= lambda_max / 1024.
                           Supported by the level-sums, multi-level, estimate
                           and path entry points; the graph, server, density
                           and trace entry points return MLMC_EINVAL for it. */
} mlmc_params;

/* Fill *p with the 600 m neutral boundary-layer scenario: u* = 0.2, f = 1e-4,
 * H = 600, kappa_sigma = 1.3, kappa_tau = 0.5, c_f = 15, eps_reg = 1e-3 H,
 * z0 = 0.1 H with w0 ~ N(0, sigma_w(z0)^2), T = 600 s, M0 = 8, levels 0..10,
 * threshold 0.1 H, FP32 paths.  Returns MLMC_OK. */
int mlmc_params_default(mlmc_params* p);

/* ---------------------------------------------------------------- results */
/* Per-level sums (Eq. Yhatell): for QoI q (0: z(T); 1: 1[z(T) < threshold] or
 * the smoothed interval P^{r,delta}_{[a,b]}(z(T)), per qoi1_mode)
 * sum[q] = { sum Y, sum Y^2, sum P_f, sum P_f^2, sum P_c, sum P_c^2 } with
 * Y = P_f - P_c (Y = P_f and P_c = 0 on level_min).  FP64, Kahan-compensated
 * within thread blocks and reduced across blocks in a fixed order. */
typedef struct mlmc_level_result {
  uint64_t n;           /* finite path pairs in the sums                        */
  uint64_t path_steps;  /* integrator steps executed (fine + coarse), all pairs */
  uint64_t n_nonfinite; /* pairs excluded because a path diverged               */
  uint64_t reserved;
  double sum[2][6];
} mlmc_level_result;

#define MLMC_MAX_LEVELS 32
typedef struct mlmc_result {
  double estimate[2];            /* MLMC estimate of E[P] per QoI              */
  double est_variance[2];        /* sum_l V_l / N_l per QoI                     */
  int32_t L;                     /* finest level used                           */
  int32_t converged;             /* 1 if the bias test passed                   */
  uint64_t N[MLMC_MAX_LEVELS];   /* samples per level (index = level)           */
  double V[MLMC_MAX_LEVELS];     /* sample variance of Y_l, QoI 0               */
  double mean_y[MLMC_MAX_LEVELS];/* sample mean of Y_l, QoI 0                   */
  uint64_t total_path_steps;
  uint64_t n_nonfinite;
  double seconds;                /* wall time of the call                       */
} mlmc_result;

/* A batch entry for the multi-level launch: `count` pairs of `level` with
 * global path indices [first, first + count). */
typedef struct mlmc_level_request {
  int32_t level;
  int32_t reserved;
  uint64_t first;
  uint64_t count;
} mlmc_level_request;

/* --------------------------------------------------------------- queries */
const char* mlmc_strerror(int code);

/* Library and device facts: out[0] = SM count, out[1] = compute capability
 * (major * 10 + minor), out[2] = library version.  Returns MLMC_ENODEV if no
 * device is visible. */
int mlmc_device_info(int32_t out[3]);

/* Tuning of the level-sums and persistent multi-level kernels for one
 * (integrator, precision): `variant` selects the compiled kernel: 1 (uncapped), 3 or 4
 * = one path pair per thread, compiled for that many resident blocks per
 * SM; 12 or 13 = two path pairs per thread on the packed FP32
 * instructions, compiled for 2 or 3 blocks per SM (FP32 only; per-path
 * results bit-identical to the one-pair kernels); FP64 only 1;
 * `items_per_block` the planner's work items per resident block (1..1024;
 * smaller items balance better, larger ones reduce per-item overhead);
 * `blocks_per_sm` the resident blocks per SM launched (0 = all that fit).
 * The table is process-wide; the library starts from GB300-measured
 * defaults and the package's autotuner replaces them.  mlmc_get_tuning
 * returns {variant, items_per_block, blocks_per_sm}.  The paper has no
 * counterpart (launch configuration only; results change only by the FP64
 * rounding of the regrouped sums). */
int mlmc_set_tuning(int integrator, int precision, int variant, int items_per_block,
                    int blocks_per_sm);
int mlmc_get_tuning(int integrator, int precision, int32_t out[3]);

/* Smallest level of the hierarchy on which `integrator` is stable for this
 * scenario: for symplectic Euler the first l with h_l lambda_max < 2
 * (Section 3.1, h < 2 / lambda(X); lambda is largest at the regularisation
 * height), else 0.  Pure host computation; MLMC_EINVAL for bad parameters. */
int mlmc_stable_level_min(const mlmc_params* p, int integrator, int32_t* level);

/* Bytes of device workspace that every entry point below needs for a batch
 * of up to `max_requests` level requests (1 for single-level calls).  The
 * workspace must be 256-byte aligned.  Pure host computation. */
size_t mlmc_workspace_bytes(const mlmc_params* p, int max_requests);

/* ------------------------------------------------------------ estimation */
/* Sums of N coupled pairs of `level` (plain paths on level_min), paths
 * [path_offset, path_offset + N); Section 3.3, Eq. (Yhatell).  Launches the
 * coupled-level kernel (the variant the tuning table names) and the
 * fixed-order reduction on `stream`, copies the sums into *out and
 * synchronises the stream.  Returns MLMC_ENONFINITE (with
 * valid *out) if any pair diverged, MLMC_EUNSTABLE for an unstable SE level
 * unless p->allow_unstable. */
int mlmc_level_sums(int level, uint64_t N, int integrator, const mlmc_params* p,
                    uint64_t seed, uint64_t path_offset, void* workspace, size_t ws_bytes,
                    void* stream, mlmc_level_result* out);

/* As mlmc_level_sums, for many levels in ONE persistent launch: blocks take
 * fixed-size work items (largest per-path cost first) from an atomic queue;
 * each item's block partial goes to its own slot and the slots of a request
 * are reduced in item order, so the sums do not depend on scheduling.
 * d_out: device array of n_req results.  No synchronisation. */
int mlmc_multilevel_sums_async(const mlmc_level_request* reqs, int n_req, int integrator,
                               const mlmc_params* p, uint64_t seed, void* workspace,
                               size_t ws_bytes, void* stream, mlmc_level_result* d_out);

/* Same, with host requests and host results (copies in, launch, copy out,
 * synchronise): the end-to-end form of the batched launch. */
int mlmc_multilevel_sums(const mlmc_level_request* reqs, int n_req, int integrator,
                         const mlmc_params* p, uint64_t seed, void* workspace,
                         size_t ws_bytes, void* stream, mlmc_level_result* out);

/* The work-item plan of a batched launch, for inspection and tests (host
 * only: no device call, no GPU needed).  `grid` is the launch's block count
 * (SMs x resident blocks per SM of the tuned variant); the tuning table
 * gives the variant and the items per block (a batch with adaptive
 * timesteps runs its own kernel: one pair per thread, 4 items per block,
 * whatever the table says).  For entry k of the launch
 * order (finest level first, stable), out[5k .. 5k + 4] = {index of the
 * request in reqs, paths per item, items, first item, single}.  Items hold
 * whole passes of a block over its pairs: 256 pairs on a one-pair kernel,
 * 512 on a packed one (two pairs per thread, variants 12 and 13), 256 again
 * for a request the packed kernel runs one pair per thread (single = 1).
 * A request goes single when one of its pairs alone is at least a quarter of
 * a thread's average work (total path-steps / (grid * 256)): such pairs set
 * the launch's length, and one pair per thread needs about two thirds of a
 * packed warp's instructions per step.  Either way every pair is the same
 * bit for bit; only the FP64 rounding of the sums' grouping changes.  Errors as
 * mlmc_multilevel_sums (MLMC_EINVAL for bad requests, grid < 1 or a batch
 * that no split into at most 32768 items covers). */
int mlmc_multilevel_plan(const mlmc_level_request* reqs, int n_req, int integrator,
                         const mlmc_params* p, int grid, uint32_t* out);

/* The batched launch of mlmc_multilevel_sums_async for callers that cannot
 * allocate device memory at all: a framework that owns every byte of device
 * memory through its own pool, a latency-bound loop that must never call
 * cudaMalloc (it can synchronise the whole device), or an embedded host with
 * a fixed memory budget.  The paper has no counterpart; this is an interface
 * convenience.
 *
 * Instead of a caller workspace it uses one array of device memory that the
 * library defines statically: 256 + 4096 * 128 bytes (about 0.5 MiB), held
 * on every GPU that loads the library until the process exits.  The work is
 * split into the same items as mlmc_multilevel_sums_async uses whenever that
 * split has at most 4096 items (the sums are then bit-identical); a larger
 * split gets larger items until it fits; a batch that cannot be split that
 * way (more than about 4096 * 2^31 pairs) returns MLMC_EWORKSPACE, more than
 * 32 requests MLMC_EINVAL.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * The first call in each CUDA context (normally a device's primary context)
 * looks up the array's device address once (cudaGetSymbolAddress, with that
 * context current; with no context current it creates the primary one) and
 * keeps it under the context's unique id, so a call after cudaDeviceReset or
 * in another context looks it up again; make the first call in a context
 * before any stream capture begins.  All calls share the one array and it
 * keeps the last call's contents: the call clears the work counter itself,
 * but two calls that overlap on the GPU (different streams, no ordering
 * between them) race on the array, so order them on one stream or with
 * events.  Arguments, results and ordering rules otherwise as
 * mlmc_multilevel_sums_async: reqs in non-increasing level order, d_out a
 * device array of n_req results, no synchronisation. */
int mlmc_multilevel_sums_noalloc(const mlmc_level_request* reqs, int n_req, int integrator,
                                 const mlmc_params* p, uint64_t seed, void* stream,
                                 mlmc_level_result* d_out);

/* Adaptive MLMC estimate of E[z(T)] to RMSE eps (Section 3.3 and the
 * sample-size rule of Giles 2008 the paper adopts in Section 6): levels are
 * added from level_min, N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k
 * C_k)), converged when max(|Yhat_{L-1}| / 2, |Yhat_L|) < eps / sqrt(2).
 * Host-driven loop on `stream`: each pass (the new level's n_init samples,
 * then the top-up of every level) is one mlmc_multilevel_sums launch over
 * the levels that need samples. */
int mlmc_estimate(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                  void* workspace, size_t ws_bytes, void* stream, mlmc_result* out);

/* mlmc_estimate sharded over `world` ranks (one per GPU; the paper has no
 * counterpart: paths are independent and keyed by global index, so any
 * split gives the same samples).  In every pass rank `rank` integrates its
 * contiguous slice of each level's new path range [N_done, N_done + dN) on
 * its own device, and calls reduce(buf, n, ctx) once, which must replace the
 * n doubles of buf by their element-wise sum over all ranks (an all-reduce,
 * called by every rank in the same order) and return 0.  buf holds per level
 * the pair count, the diverged count, the steps, the twelve FP64 sums and,
 * in the last slot, an error flag: a rank whose launch failed still joins
 * the reduction, and then every rank returns its error (MLMC_ECOMM on the
 * others).  All ranks then apply the same N_l and bias-test decisions, so
 * they return the same result, equal to mlmc_estimate's up to the FP64
 * rounding of the cross-rank sum.  world = 1 needs no hook.  A hook that
 * returns non-zero gives MLMC_ECOMM. */
typedef int (*mlmc_allreduce_fn)(double* buf, int n, void* ctx);
int mlmc_estimate_sharded(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                          int rank, int world, mlmc_allreduce_fn reduce, void* ctx,
                          void* workspace, size_t ws_bytes, void* stream, mlmc_result* out);

/* The host-driven estimate one pass at a time, for checkpoint and resume.
 * The driver's whole state is the plain struct below (no pointers): it can
 * be copied, written to a file and read back in another process, and a run
 * resumed from it continues exactly as the uninterrupted one, because every
 * pass's launch depends only on the state (path indices continue from
 * n_done, the RNG is keyed by path index).
 *   mlmc_estimate_begin   validates the arguments and starts a state at
 *                         level_min (no device work)
 *   mlmc_estimate_pass    runs the next pass -- the new level's n_init
 *                         samples, or the top-up of every level to Eq. 12's
 *                         N_l followed by the bias test -- as one
 *                         mlmc_multilevel_sums launch on `stream`, and
 *                         synchronises it; returns 1 once the estimate is
 *                         complete (then does nothing), MLMC_OK while passes
 *                         remain, or an error (the state is then unchanged)
 *   mlmc_estimate_result  the result of the state (any time; final once
 *                         complete), with mlmc_estimate's return codes
 * mlmc_estimate runs exactly these steps, so the three give its result bit
 * for bit. */
typedef struct mlmc_estimate_state {
  double eps;                                   /* RMSE target                   */
  uint64_t seed;
  int32_t integrator;
  int32_t L;                                    /* finest level so far           */
  int32_t phase;                                /* 0 new level next, 1 top-up
                                                   next, 2 complete              */
  int32_t converged;                            /* 1 if the bias test passed     */
  uint64_t n_done[MLMC_MAX_LEVELS];             /* samples issued per level      */
  uint64_t n[MLMC_MAX_LEVELS];                  /* finite pairs in the sums      */
  uint64_t n_nonfinite[MLMC_MAX_LEVELS];
  uint64_t path_steps[MLMC_MAX_LEVELS];
  double sum[MLMC_MAX_LEVELS][2][6];            /* as mlmc_level_result.sum      */
  double seconds;                               /* wall time of the passes run   */
  int32_t passes;                               /* passes run                    */
  int32_t reserved;
} mlmc_estimate_state;
int mlmc_estimate_begin(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                        mlmc_estimate_state* st);
int mlmc_estimate_pass(mlmc_estimate_state* st, const mlmc_params* p, void* workspace,
                       size_t ws_bytes, void* stream);
int mlmc_estimate_result(const mlmc_estimate_state* st, const mlmc_params* p, mlmc_result* out);

/* The same adaptive estimate with the whole loop on the device, as one CUDA
 * graph: an init kernel, then a conditional while-node whose body is the
 * persistent multi-level kernel over the levels that need samples, the
 * fixed-order per-level reduction, and a one-warp update kernel that adds
 * the sums, applies N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k)),
 * the bias test and the next plan, and sets the loop condition.  The driver
 * state, plan and result live in the workspace (which must stay alive and
 * unused by other calls while the graph runs).  The loop is bounded: after
 * its pass limit (4 * MLMC_MAX_LEVELS passes; mlmc_graph_create_ex sets a
 * smaller one) a pass that would start another one ends the loop instead,
 * and mlmc_graph_result returns MLMC_ETIMEOUT with the partial result.
 *   mlmc_graph_create   builds and instantiates the graph (host work; no
 *                       kernel runs yet; two pinned host buffers, about
 *                       5 KB, receive the result of each launch); returns
 *                       an opaque handle
 *   mlmc_graph_launch   enqueues one complete estimate on `stream`
 *   mlmc_graph_result   copies the result of the last launch into *out and
 *                       synchronises `stream`; same codes as mlmc_estimate
 *   mlmc_graph_destroy  frees the handle (host resources only)
 * mlmc_estimate_graph does all four once (without the pinned buffers, whose
 * allocation would cost more than they save on a single launch).  The
 * graph's estimate equals
 * mlmc_estimate's up to the FP64 rounding of the level sums (the batched
 * kernel groups paths into items differently). */
typedef struct mlmc_graph_s* mlmc_graph;
int mlmc_graph_create(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                      void* workspace, size_t ws_bytes, mlmc_graph* out);
/* mlmc_graph_create with the device loop's pass limit: max_passes launches of
 * the persistent kernel at most (1..4 * MLMC_MAX_LEVELS; 0 = that default),
 * after which the update kernel ends the loop with MLMC_ETIMEOUT.  A watchdog
 * on the device-side loop, settable from the host; the paper has no
 * counterpart. */
int mlmc_graph_create_ex(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                         int max_passes, void* workspace, size_t ws_bytes, mlmc_graph* out);
int mlmc_graph_launch(mlmc_graph g, void* stream);
int mlmc_graph_result(mlmc_graph g, void* stream, mlmc_result* out);
int mlmc_graph_destroy(mlmc_graph g);
int mlmc_estimate_graph(double eps, int integrator, const mlmc_params* p, uint64_t seed,
                        void* workspace, size_t ws_bytes, void* stream, mlmc_result* out);

/* Plain Monte Carlo (Eq. StMCestimator) at `level`'s timestep to RMSE eps:
 * n_pilot paths estimate Var[P], then N = ceil(2 Var / eps^2) in total. */
int mlmc_stmc_estimate(double eps, int level, int n_pilot, int integrator,
                       const mlmc_params* p, uint64_t seed, void* workspace,
                       size_t ws_bytes, void* stream, mlmc_result* out);

/* ------------------------------------------------------- binned density */
/* The concentration field of Section 6.3 (Eq. vector_QoI): k equal bins
 * [i H / k, (i + 1) H / k), i < k <= 32, each QoI the smoothed interval
 * P^{r,delta} of its bin (order p->smooth_r, width p->smooth_delta > 0).
 * mlmc_level_pdf_sums: N pairs of `level` from path_offset; out[2i] = sum
 *   Y_i, out[2i + 1] = sum Y_i^2 (host array of 2k doubles), *n_ok finite
 *   pairs, *n_nonfinite diverged pairs; synchronises the stream.
 * mlmc_estimate_pdf: adaptive MLMC estimate of the k bin probabilities to
 *   RMSE eps per bin, N_l chosen with max_i Var[Y_{l,i}] (Section 6.3) and
 *   the bias test applied to every bin; pdf[i] (host, k doubles) gets bin
 *   i's estimate; *out as mlmc_estimate with estimate[0] = sum_i pdf[i],
 *   est_variance[0] the largest per-bin estimator variance, V[l] the largest
 *   per-bin variance of level l. */
int mlmc_level_pdf_sums(int level, uint64_t N, int integrator, const mlmc_params* p,
                        uint64_t seed, uint64_t path_offset, int k, void* workspace,
                        size_t ws_bytes, void* stream, double* out, uint64_t* n_ok,
                        uint64_t* n_nonfinite);
int mlmc_estimate_pdf(double eps, int integrator, const mlmc_params* p, uint64_t seed, int k,
                      void* workspace, size_t ws_bytes, void* stream, double* pdf,
                      mlmc_result* out);

/* ------------------------------------------------------------- serving */
/* A continuous-batching server of dispersion queries (the operational use
 * the paper's introduction motivates).  Each query is an adaptive MLMC
 * estimate (the rule of mlmc_estimate) of its own scenario and tolerance;
 * its Philox stream is p->stream_id, the key is the server's seed.
 *
 * Device state.  An admitted query owns a record in a pool that the server
 * carves from the caller's workspace: its Model and its whole per-level
 * state -- for every level level_min..L_max the twelve FP64 sums, the pair,
 * diverged and step counts, the samples folded and the pass targets -- and
 * the driver's level, pass and plan.  After each launch a fold kernel adds
 * every chunk's sums into its query's record and, once a pass is complete,
 * applies Eq. 12's sample sizes and the bias test on the device; the host
 * reads back only each touched query's plan (the samples of its next pass)
 * or, when it is done, its result.
 *
 * Admission is by memory: a queued query is admitted, in arrival order,
 * when a record of its size -- mlmc_server_query_bytes(p), which grows with
 * its number of levels -- fits in the free part of the pool (first fit; the
 * head of the queue is never overtaken) and fewer than max_active queries
 * are active.  A query whose record exceeds the whole pool is refused at
 * submit (MLMC_EWORKSPACE).
 *
 *   mlmc_server_workspace_bytes  device workspace: the launch buffers plus a
 *                                pool of max_active records of 17 levels
 *                                (0 gives the launch buffers alone; any
 *                                larger workspace is all pool)
 *   mlmc_server_query_bytes      bytes of one query's record
 *   mlmc_server_create   binds the workspace; work queued on `stream`
 *                        before the call is ordered before the server's
 *                        launches, which run on four streams of its own, the
 *                        folds on a fifth; allocates those streams, their
 *                        events and pinned host staging buffers (no device
 *                        memory)
 *   mlmc_server_submit   validates and queues a query; returns its id
 *   mlmc_server_tick     takes the plans of the launches whose folds have
 *                        completed (oldest first), admits queued queries
 *                        while their records fit, and puts one more launch
 *                        in flight (at most four): one persistent launch
 *                        (of the one-pair kernel, variant 4, whatever the
 *                        tuning table holds: the finest work items) over
 *                        chunks (at most 2^26 path-steps each) of the
 *                        active queries' pending passes -- least pending
 *                        work first, a waiting query's priority doubling
 *                        every launch -- up to 2^28 path-steps, 2048
 *                        requests and 32768 work items, holding only pairs
 *                        at most 4 times as long as its first chunk's (or
 *                        2048 path-steps), followed by its fold; when all
 *                        four are in flight, or nothing is left to issue, it
 *                        first waits for the oldest.  n_done: queries
 *                        finished in this call; n_active: queries left
 *                        (active and queued).  After a CUDA error every
 *                        later call returns that error (launches in flight
 *                        may be lost)
 *   mlmc_server_poll     1 while the query runs; its final status (MLMC_OK,
 *                        MLMC_ENOTCONV, MLMC_ENONFINITE) with the result and
 *                        its submit-to-finish latency once done
 *   mlmc_server_release  forgets a finished query
 *   mlmc_server_stats    out = {ticks, finished, path-steps, busy seconds,
 *                        active, queued}
 *   mlmc_server_pool     out = {record bytes in use, pool bytes}
 * A pass's chunks, their split into work items and their folding order
 * depend only on the query (and the server's grid), so a query's result is
 * bitwise the same alone and in any mix; the scheduling decides only when a
 * chunk runs.  mlmc_server_destroy waits for the launches in flight. */
typedef struct mlmc_server_s* mlmc_server;
size_t mlmc_server_workspace_bytes(int max_active);
size_t mlmc_server_query_bytes(const mlmc_params* p);
int mlmc_server_create(int integrator, int precision, int max_active, uint64_t seed,
                       void* workspace, size_t ws_bytes, void* stream, mlmc_server* out);
int mlmc_server_submit(mlmc_server s, const mlmc_params* p, double eps, uint64_t* query_id);
int mlmc_server_tick(mlmc_server s, int* n_done, int* n_active);
int mlmc_server_poll(mlmc_server s, uint64_t query_id, mlmc_result* out, double* latency_s);
int mlmc_server_release(mlmc_server s, uint64_t query_id);
int mlmc_server_stats(mlmc_server s, double out[6]);
int mlmc_server_pool(mlmc_server s, uint64_t out[2]);
int mlmc_server_destroy(mlmc_server s);

/* ---------------------------------------------------------- path outputs */
/* Final states of N pairs of `level` into d_states (N x 4 values of the path
 * precision: z_f, w_f, z_c, w_c; coarse entries 0 on level_min) and
 * d_flags (N int32: bit 0 diverged).  No synchronisation. */
int mlmc_level_paths_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                           uint64_t seed, uint64_t path_offset, void* d_states,
                           int32_t* d_flags, void* stream);

/* mlmc_level_paths_async through the path code of one tuning variant of the
 * level-sums and persistent multi-level kernels (see mlmc_set_tuning):
 * variant 0 = the variant the tuning table names for (integrator,
 * precision); 1, 3, 4 = one pair per thread at that register budget; 12, 13
 * = two pairs per thread on the packed FP32 instructions (thread g takes
 * pairs 2g and 2g + 1; for an odd N the last lane is computed and
 * discarded), the code the batched launches reduce.  Every variant gives the
 * same paths bit for bit; this entry point lets a caller check that, and
 * check the batched kernels pair by pair.  Same outputs and layout as
 * mlmc_level_paths_async; MLMC_EINVAL for another variant, or a packed one
 * with FP64 paths.  With adaptive timesteps every variant runs the one
 * adaptive kernel.  No synchronisation.  Paths as Section 3.3 (Eqs.
 * MethodSymplecticEuler, MethodSymplecticEulerOU, MethodBAOAB and the coupled
 * increments of Eqs. euler_coupled_treatment, splitting_coupled_treatment). */
int mlmc_level_paths_variant_async(int variant, int level, uint64_t N, int integrator,
                                   const mlmc_params* p, uint64_t seed, uint64_t path_offset,
                                   void* d_states, int32_t* d_flags, void* stream);

/* mlmc_level_paths_async for adaptive timesteps (p->z_adapt > 0, else
 * MLMC_EINVAL), also writing the integrator steps of each pair: d_steps gets
 * N x 2 int64 values (fine, coarse; coarse 0 on level_min).  No
 * synchronisation. */
int mlmc_level_paths_steps_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                                 uint64_t seed, uint64_t path_offset, void* d_states,
                                 int32_t* d_flags, int64_t* d_steps, void* stream);

/* Full trajectories of N pairs (meant for small N): d_trace_f gets N x (M+1)
 * x 3 values (z, w, S per fine time point), d_trace_c N x (M/2+1) x 3 (may be
 * NULL on level_min).  Uniform timesteps only.  No synchronisation. */
int mlmc_path_trace_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                          uint64_t seed, uint64_t path_offset, void* d_trace_f,
                          void* d_trace_c, void* stream);

/* BAOAB's state after the first half of every step (Eq. MethodBAOAB: after
 * the B and A half-steps and the fold that follows, where the step's noise
 * enters): d_half_f gets N x M x 3 values (z, w, S; row n for fine step n),
 * d_half_c N x M/2 x 3 (may be NULL on level_min).  Together with
 * mlmc_path_trace_async it locates every fold of a path; a reflection whose
 * order FP32 and FP64 paths disagree on shows here even when the full-step
 * parities agree again.  BAOAB with uniform timesteps only (else
 * MLMC_EINVAL).  No synchronisation. */
int mlmc_path_trace_half_async(int level, uint64_t N, int integrator, const mlmc_params* p,
                               uint64_t seed, uint64_t path_offset, void* d_half_f,
                               void* d_half_c, void* stream);

/* ------------------------------------------------------------ measurement */
/* The paper has no counterpart: this measures the roofline denominator of
 * the path kernels.  Runs a kernel of independent FP32 FMA chains (8 per
 * thread, `iters` iterations, every SM fully occupied) on `stream`, times it
 * with CUDA events and writes the achieved FP32 rate in FLOP/s (FMA = 2) to
 * *flops_per_s.  d_scratch: at least 4 MB of device memory that receives
 * the chain results.  Synchronises the stream. */
int mlmc_fp32_peak_probe(int iters, void* d_scratch, void* stream, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_GB300_H */
