/*
 * hc.h -- C ABI of the GB300 (sm_103a) hot path of the multithreaded path tracker of
 * Verschelde & Yoffe, "Quality Up in Polynomial Homotopy Continuation by Multithreaded
 * Path Tracking" (2011).
 *
 * The library evaluates a sparse polynomial system and its full Jacobian by
 * algorithmic differentiation (Sec. 6), in complex double, double-double or
 * quad-double arithmetic (Sec. 1, 2), assembles the homotopy
 *     h(x,t) = gamma (1-t) g(x) + t f(x),   g_i(x) = x_i^{d_i} - 1,
 * with t a parameter (Sec. 7, Table 6 caption), and runs the Newton corrector of
 * Alg. 4.1 (Gaussian elimination with partial pivoting, Sec. 4) and the path tracker
 * of Alg. 3.1 on top of it.
 *
 * Conventions shared by every call:
 *   - L = number of limbs per real: 1 (double), 2 (double-double), 4 (quad-double);
 *     a multi-limb value is the unevaluated sum of its limbs, leading limb first.
 *   - Device arrays are structure-of-arrays with the point index fastest:
 *       X[2][L][n][npts]          points (re limbs, then im limbs)
 *       F[2][L][npoly][npts]      values
 *       J[2][L][npoly][n][npts]   Jacobians, row i = polynomial, column j = variable
 *     i.e. part c, limb l, index i of point p sits at base[((c*L + l)*rows + i)*npts + p].
 *   - Return codes: HC_SUCCESS (0) or a negative HC_E* code; hc_last_error() then
 *     describes the failure.  Per-point outcomes go to caller-owned status arrays.
 *   - All device calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  Calls on the same hc_system share its
 *     workspace and must not overlap in time: issue them on one stream.
 *   - The caller owns every input/output buffer; the library owns hc_system and its
 *     device tables and workspace.
 *   - Invalid arguments are rejected on the host with HC_EINVAL before any launch.
 */
#ifndef HC_H
#define HC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define HC_SUCCESS 0
#define HC_EINVAL (-1)    /* invalid argument or malformed system */
#define HC_ENOMEM (-2)    /* device allocation failed */
#define HC_ECUDA (-3)     /* a CUDA runtime call failed */
#define HC_ENOTIMPL (-4)  /* combination not supported */
#define HC_ETIMEOUT (-5)  /* a bounded device-side wait ran out */

/* per-point / per-path status */
#define HC_OK 0         /* converged / tracked to t = 1 */
#define HC_NOCONV 1     /* end-point Newton did not reach its tolerance */
#define HC_SINGULAR 2   /* a pivot of the elimination was exactly zero */
#define HC_MIN_STEP 3   /* step size fell below its minimum (Alg. 3.1 stop criterion) */
#define HC_MAX_STEPS 4  /* corrector stages exhausted (Alg. 3.1 stop criterion) */
#define HC_DIVERGED 5   /* ||x||_inf exceeded its bound */
#define HC_NONFINITE 6  /* Inf or NaN met */

/* precision = limbs per real */
#define HC_PREC_D 1
#define HC_PREC_DD 2
#define HC_PREC_QD 4

/* linear solve of the Newton step */
#define HC_LU_NATIVE 0       /* elimination in the working precision (Sec. 4) */
#define HC_LU_FP64_REFINE 1  /* FP64 LU, residual and update in the working precision */

typedef struct hc_system hc_system;

/*
 * hc_system_load -- validate a sparse system and upload it to the current device.
 * The normalised monomial form of Sec. 6: polynomial i owns monomials
 * mon_ptr[i] .. mon_ptr[i+1]-1; monomial m owns variables var_ptr[m] .. var_ptr[m+1]-1
 * with strictly increasing 0-based indices var_idx[] < n and exponents var_exp[] >= 1;
 * a monomial with no variables is a constant term.  At most 32 variables per monomial,
 * exponents at most 64, n at most 1024.
 *   coef   host, [nmon][2][L] doubles (re limbs, im limbs), finite
 *   prec   HC_PREC_D / _DD / _QD (= L)
 *   gamma  host, the homotopy constant (re, im) in double
 * The degree d_i of the start system is the largest total degree of a monomial of f_i.
 * All host arrays are copied; the caller keeps ownership.  Returns HC_SUCCESS and
 * *out, or HC_EINVAL (malformed input, nothing allocated), HC_ENOMEM, HC_ECUDA.
 */
int hc_system_load(hc_system **out, int n, int npoly, const int32_t *mon_ptr,
                   const int32_t *var_ptr, const int32_t *var_idx, const int32_t *var_exp,
                   const double *coef, int prec, const double gamma[2]);

/* Free a system and its device tables and workspace (NULL is a no-op).  Synchronises
 * the device first, so no call may still be using it. */
void hc_system_free(hc_system *sys);

/* Sizes of a loaded system: any pointer may be NULL.  Returns HC_EINVAL on NULL sys. */
int hc_system_info(const hc_system *sys, int *n, int *npoly, int *nmon, int *nvar,
                   int *prec, int *max_exp, int *max_deg);

/*
 * hc_eval_jac -- values and full Jacobian at npts points (Alg. 4.1 Monomial_Evaluation
 * followed by Coefficient_Product; the monomial scheme of Sec. 6), per term or with
 * shared monomials (hc_system_set_eval_mode; the same values up to rounding).
 *   t < 0   evaluate f itself (npoly may differ from n);
 *   t >= 0  evaluate the homotopy h(., t) and its Jacobian in x (requires npoly == n
 *           and every d_i >= 1).
 *   x  device X[2][L][n][npts];  f  device F[2][L][npoly][npts];
 *   J  device J[2][L][npoly][n][npts], or NULL for values only.
 * Uses the system's workspace (allocated on first use, grown as needed): the power table
 * and, in the shared-monomial scheme when npts / 32 tiles give the GPU fewer than about 8
 * warps per SM, the partial sums of G groups of distinct monomials (G up to 64:
 * G * 2 * L * npoly * (1 + n) doubles per point, about 2 GB in all for Table 1's
 * 40 x 40 system in DD, whatever npts).
 * npts == 0 is a no-op.  Errors: HC_EINVAL, HC_ENOMEM, HC_ECUDA.
 */
int hc_eval_jac(hc_system *sys, int npts, double t, const double *x, double *f, double *J,
                void *stream);

/*
 * hc_newton_step -- one Newton iteration of Alg. 4.1 at every point, on h(., t)
 * (t >= 0) or on f (t < 0, npoly == n required):
 *   evaluate h and J at x; res_norm[p] = max_i |h_i| (moduli of the leading limbs,
 *   in double) at the incoming x; solve J dz = -h with partial pivoting; x += dz.
 *   lu_mode     HC_LU_NATIVE or HC_LU_FP64_REFINE
 *   max_refine  refinement sweeps for HC_LU_FP64_REFINE (>= 1); refinement stops
 *               early once ||correction||_inf <= 2^(-53 L) max(||x||_inf, ||dz||_inf),
 *               or when a correction is no smaller than the previous one, which is
 *               then not applied (norms of the leading limbs)
 *   x        device X[2][L][n][npts], updated in place where status is HC_OK
 *   res_norm device double[npts] (may be NULL)
 *   status   device int32[npts]: HC_OK, HC_SINGULAR (x unchanged) or HC_NONFINITE
 *            (x unchanged)
 *   sweeps   device int32[npts] (may be NULL): refinement sweeps taken (0 for native)
 * Uses the system's workspace: that of hc_eval_jac plus h, J and the solve's arrays.
 * Errors: HC_EINVAL, HC_ENOMEM, HC_ECUDA.
 */
int hc_newton_step(hc_system *sys, int npts, double t, double *x, int lu_mode,
                   int max_refine, double *res_norm, int32_t *status, int32_t *sweeps,
                   void *stream);

/*
 * hc_set_tiles -- tile shape of the per-term evaluation kernel for every later call in
 * this process (the autotuner's knob; 0 = automatic):
 *   rows_per_task  polynomials one warp evaluates per task (its 32 points each)
 *   blocks_per_sm  resident 4-warp blocks per SM of the persistent grid (<= 32)
 * Process-wide host-side setting, not synchronised with calls in other threads; any
 * setting gives the same results bit for bit.  Errors: HC_EINVAL.
 */
int hc_set_tiles(int rows_per_task, int blocks_per_sm);

/*
 * hc_set_track_tiles -- execution shape of hc_track_path / hc_track_resume for every
 * later call in this process (the tracker autotuner's knobs; 0 = automatic):
 *   threads_per_block  threads of a path's block: 64, 128 (automatic), 256 or 512 (double
 *                      and DD; QD runs 512 as 256); the register budget per thread stays
 *                      that of 512 (double, DD) or 384 (QD) threads per SM
 *   blocks_per_sm      path blocks resident per SM, at most what occupancy allows
 *   factors            0 or 1: the FP64 factors of a path in shared memory when a block's
 *                      share of the SM holds them (else global memory); 2: always global
 *   grid_chunk         contributions per chunk of an entry's sum in HC_TRACK_GRID (32)
 * Results do not depend on threads_per_block, blocks_per_sm or factors (bit for bit).
 * grid_chunk changes the order in which the whole-GPU engine adds an entry's
 * contributions (results within the precision's rounding).  Process-wide host-side
 * setting, not synchronised with calls in other threads.  Errors: HC_EINVAL.
 */
int hc_set_track_tiles(int threads_per_block, int blocks_per_sm, int factors, int grid_chunk);

/* The current settings of hc_set_track_tiles (any pointer may be NULL). */
int hc_get_track_tiles(int *threads_per_block, int *blocks_per_sm, int *factors, int *grid_chunk);

/* predictors (Sec. 5) and tracker execution modes */
#define HC_PRED_SECANT 0     /* linear through the last two accepted points */
#define HC_PRED_QUADRATIC 1  /* per coordinate, the parabola through the last three */
#define HC_PRED_TANGENT 2    /* Euler: x + h dx/dt with dx/dt = -J^-1 dh/dt, dh/dt = f - gamma g,
                                from the FP64 factors and the evaluation of the last Newton
                                iteration of the last accepted stage (an FP64 direction);
                                zeroth order on the first stage; not with HC_TRACK_GRID */
#define HC_TRACK_PERSISTENT 0  /* one persistent kernel, paths from an atomic queue */
#define HC_TRACK_GRAPH 1       /* one stage per launch, replayed as a CUDA graph */
#define HC_TRACK_GRID 2        /* one path at a time on the whole GPU: each stage a CUDA
                                  graph of grid-wide and single-block kernels (for
                                  systems of ~1e5 monomials; HC_LU_FP64_REFINE only) */

/* Options of hc_track_path.  The paper gives no constants (Alg. 3.1); the defaults of
 * hc_track_opts_default follow Tables 2-3: steps lambda0 * 2^j. */
typedef struct {
    double lambda0;     /* first step size, 0.01 */
    double lambda_min;  /* stop (HC_MIN_STEP) once the step falls below this, 1e-12 */
    double lambda_max;  /* largest step, 0.08 (= lambda0 * 2^3) */
    double grow;        /* step factor after grow_after consecutive successes, 2 */
    double shrink;      /* step factor after a failed corrector stage, 0.5 */
    double eps;         /* corrector converged: ||h||_inf <= eps ...                */
    double eps_x;       /*   ... or ||dz||_inf <= eps_x max(1, ||z||_inf)           */
    double eps_end;     /* the same two tolerances for the end game at t = 1        */
    double eps_end_x;
    double div_bound;   /* ||z||_inf above this ends the path as HC_DIVERGED, 1e6 */
    int32_t max_it;     /* Newton iterations per corrector stage, 3 */
    int32_t end_it;     /* Newton iterations of the end game, 8 */
    int32_t grow_after; /* consecutive successes before the step grows, 3 */
    int32_t max_steps;  /* corrector stages before HC_MAX_STEPS, 100000 */
    int32_t predictor;  /* HC_PRED_SECANT, HC_PRED_QUADRATIC or HC_PRED_TANGENT */
    int32_t lu_mode;    /* HC_LU_NATIVE or HC_LU_FP64_REFINE */
    int32_t max_refine; /* refinement sweeps of HC_LU_FP64_REFINE, 4 */
    int32_t mode;       /* HC_TRACK_PERSISTENT or HC_TRACK_GRAPH */
    int32_t graph_steps;/* launches per graph in HC_TRACK_GRAPH, 16 */
    int32_t reserved;
    const float *proposer;   /* device, HC_MLP_NPARAM weights of the learned step
                                proposer, or NULL for the plain controller */
    double proposer_margin;  /* the proposal is lambda_last * 2^(m - margin), 0.5.  The
                                plain controller runs alongside on the same outcomes; its
                                step lambda_p bounds the proposal: after an accepted
                                stage to [max(lambda_min, lambda_p / 4), lambda_max],
                                after a rejection to at most shrink * the step that
                                failed, and MIN_STEP when that is below lambda_min */
    double explore;          /* for collecting the proposer's training data: the next step
                                of the plain controller times 2^u, u uniform in
                                [-explore, explore], clamped to [lambda_min, lambda_max];
                                u from SplitMix64 (Steele, Lea & Flood 2014) of
                                explore_seed ^ (path index << 32) ^ stage count.  0 (the
                                default) = off; ignored with a proposer */
    uint64_t explore_seed;
} hc_track_opts;

/* Per-path result (the statistics of Tables 2-3). */
typedef struct {
    int64_t n_succ;      /* successful corrector stages */
    int64_t n_corr;      /* corrector stages */
    int64_t newton_its;  /* Newton iterations along the path (end game excluded) */
    double min_step, avg_step;  /* over accepted stages */
    double t_end;        /* t reached */
    double res_end;      /* residual of the last end-game iteration (-1: none) */
    int32_t status;      /* HC_OK, HC_NOCONV, HC_SINGULAR, HC_MIN_STEP, ... */
    int32_t end_its;     /* Newton iterations of the end game */
} hc_path_stats;

/* The state of one path between corrector stages: what hc_track_resume saves and
 * restarts from (checkpoint / resume; the paper has no such feature, its tracker keeps
 * these values in the variables of Alg. 3.1).  The two accepted points before the
 * current one live in the caller's hist buffer (see hc_track_resume).  A caller may
 * inspect the state, store it, or change it between calls: e.g. to continue a path that
 * stopped at HC_MAX_STEPS, raise opts->max_steps and set phase = 1, status = HC_OK. */
typedef struct {
    double t;          /* t of the current point (the last accepted one) */
    double tp, tpp;    /* t of the two accepted points before it */
    double lambda;     /* step of the next corrector stage */
    double minstep;    /* smallest accepted step (+inf before the first) */
    double sumstep;    /* sum of the accepted steps */
    double res_end;    /* residual of the last end-game iteration, -1 before the end game */
    double pad;
    int64_t n_succ;    /* accepted corrector stages */
    int64_t n_corr;    /* corrector stages */
    int64_t nits;      /* Newton iterations of the stages */
    int32_t nhist;     /* accepted points in the history (current one included): 1, 2, 3 */
    int32_t consec;    /* consecutive accepted stages since the step last grew */
    int32_t status;    /* HC_OK while the path runs; its final status once done */
    int32_t phase;     /* 0: start at t = 0 from x; 1: tracking; 2: the end game is next;
                          3: done */
    int32_t end_its;   /* Newton iterations of the end game */
    int32_t pad2;
    double hl[3];      /* the last three attempted steps (latest first) } features of */
    double hr[3];      /* their last residuals                           } the learned */
    double pcd;        /* the last predictor-corrector distance (-1)     } step proposer */
    double cond;       /* log10 condition estimate of the last factorisation */
    int32_t hi[3];     /* Newton iterations of the last three stages */
    int32_t pad3;
    double lam_plain;  /* the plain controller's step, run alongside a proposer */
    int64_t pid;       /* path index: the stream of the exploration generator */
} hc_path_state;

/* One corrector stage, as logged for the learned step-size proposer. */
typedef struct {
    double t;            /* t before the stage */
    double lambda;       /* step attempted (t' - t) */
    double res_first;    /* residual of the predicted point */
    double res_last;     /* residual of the last Newton iterate evaluated */
    double pc_dist;      /* ||corrected - predicted||_inf if accepted, else -1 */
    double cond_log10;   /* log10 of max/min pivot modulus of the last factorisation */
    int32_t iters;       /* Newton iterations */
    int32_t accepted;    /* 1 if the stage was accepted */
} hc_step_record;

/* Evaluation schemes of the point kernels (hc_eval_jac, hc_newton_step). */
#define HC_EVAL_AUTO 0      /* the scheme with fewer FP64 instructions, by at least 10 % */
#define HC_EVAL_PER_TERM 1  /* each term's monomial and partials with its coefficient folded
                               into the common factor (Sec. 6) */
#define HC_EVAL_SHARED 2    /* each distinct monomial and its partials once per point, then
                               one coefficient product per term and partial: for systems
                               whose polynomials share monomials (a common support, the
                               40 x 40 system of Sec. 4 behind Table 1) */

/* Choose the evaluation scheme of sys (HC_EVAL_AUTO restores the choice made at load).
 * Both schemes compute the same values up to rounding.  No device work.  Errors:
 * HC_EINVAL for a NULL sys or an unknown mode. */
int hc_system_set_eval_mode(hc_system *sys, int mode);

/* The scheme in use (HC_EVAL_PER_TERM or HC_EVAL_SHARED), and the FP64 instructions per
 * point of each scheme's evaluation with Jacobian, counted at load with complex
 * double-double weights (either pointer may be NULL).  HC_EINVAL for a NULL sys. */
int hc_system_eval_mode(const hc_system *sys, double *ops_per_term, double *ops_shared);

/* Fill *opts with the defaults listed above. */
void hc_track_opts_default(hc_track_opts *opts);

/*
 * hc_track_path -- track npaths solution paths of h(x,t) = gamma (1-t) g(x) + t f(x),
 * g_i = x_i^{d_i} - 1, from t = 0 to t = 1 (Alg. 3.1 with the Newton corrector of
 * Alg. 4.1): predict at t' = min(t + lambda, 1), correct with at most max_it Newton
 * iterations, accept (shift the history; grow lambda after grow_after successes) or
 * step back (shrink lambda); stop on lambda < lambda_min, max_steps stages or
 * ||z|| > div_bound; fail := (t < 1).  At t = 1 an end game of at most end_it Newton
 * iterations on f.
 *   sys    host array of npaths systems (each npoly == n <= 256, degrees >= 1, all
 *          of one precision); path p runs on sys[p] (the same system may repeat)
 *   x0     device, start points packed path after path, path p at offset
 *          2 L (n_0 + ... + n_{p-1}) doubles as [2][L][n_p]
 *   x1     device, end points in the same packing (caller-owned; may not alias x0)
 *   stats  host, npaths results, valid on return
 *   log    device, npaths * log_cap records (record s of path p at p * log_cap + s),
 *          or NULL with log_cap = 0
 * One thread block per path (HC_TRACK_GRID: the whole GPU per path, paths in turn);
 * blocks take paths largest first (by the cost of a stage), the first wave in a fixed
 * shuffled order.  Each path's result does not depend on the order, the mode or the
 * other paths (bit for bit).  Synchronises the stream before returning.  Allocates and
 * frees its own workspace.  Errors: HC_EINVAL, HC_ENOMEM, HC_ECUDA, HC_ETIMEOUT (graph
 * mode only: paths still unfinished after max_steps / graph_steps + 2 replays).
 */
int hc_track_path(hc_system *const *sys, int npaths, const double *x0, double *x1,
                  const hc_track_opts *opts, hc_path_stats *stats, hc_step_record *log,
                  int log_cap, void *stream);

/*
 * hc_track_resume -- checkpoint / resume of hc_track_path (Alg. 3.1): advance each path
 * by at most max_stages corrector stages from its saved state, then run its end game if
 * it reached t = 1, and save the state again.  Repeated calls with max_stages = k give
 * the same paths, bit for bit, as one hc_track_path call (same options).
 *   sys, opts  as for hc_track_path (every mode; the tangent predictor needs the tangent
 *              of the history, so it resumes only from states this function wrote)
 *   x      device, packed as hc_track_path's x0, in/out: on input the start point of a
 *          path in phase 0, else its current point; on output its current point
 *   hist   device, in/out, 3 vectors of 2 L n_p doubles per path, path p at offset
 *          3 * 2 L (n_0 + ... + n_{p-1}): the accepted point before the current one and
 *          the one before that ([2][L][n_p] each; the first state.nhist - 1 are used),
 *          then dx/dt at the current point ([2][n_p] leading limbs in the first 2 n_p
 *          doubles; written by the tangent predictor only).  Need not be initialised for
 *          a path in phase 0.
 *   state  host, npaths states in/out (phase 0: start the path at t = 0 from x; phase 3:
 *          left as is)
 *   max_stages  >= 1, corrector stages per path in this call
 *   stats  host, npaths results as hc_track_path's (may be NULL)
 *   log    device, npaths * log_cap records of this call's stages (record s of path p at
 *          p * log_cap + s), or NULL with log_cap = 0
 * Synchronises the stream before returning.  Allocates and frees its own workspace.
 * Errors: HC_EINVAL (bad argument, an unknown phase), HC_ENOMEM, HC_ECUDA, HC_ETIMEOUT.
 */
int hc_track_resume(hc_system *const *sys, int npaths, double *x, double *hist,
                    hc_path_state *state, int max_stages, const hc_track_opts *opts,
                    hc_path_stats *stats, hc_step_record *log, int log_cap, void *stream);

/*
 * The learned step-size proposer (not in the paper; the plain controller of Alg. 3.1
 * stays the fallback and the corrector still judges every step): a 12 -> 64 -> 64 -> 1
 * perceptron with GELU, bfloat16 operands, float32 accumulation and float32 master
 * weights.  Parameters, HC_MLP_NPARAM floats: W1 (64x12, row-major) | b1 (64) |
 * W2 (64x64) | b2 (64) | W3 (64) | b3 (1).  Its output m estimates log2 of the largest
 * next step, relative to the last attempted one, that the corrector would accept.
 * Features (HC_MLP_IN floats per record, scaled to order one): t;
 * log2(lambda/lambda0)/8 of the last three attempted steps; their Newton iteration
 * counts/4; log10 of their last residuals, clipped to [-40, 5], /10; the same for the
 * last predictor-corrector distance (-4 after a rejection); the last condition estimate
 * (hc_step_record.cond_log10)/4.  Missing history: steps lambda0, 0 iterations,
 * residual and distance -4, condition 0.
 * Training loss per logged stage with attempted log2 step ratio r and outcome a:
 * z = m - r, softplus(-kappa z) if accepted else softplus(kappa z), averaged.
 * All pointers are device pointers; the calls are asynchronous on the stream.
 */
#define HC_MLP_IN 12
#define HC_MLP_NPARAM 5057

/* grad[HC_MLP_NPARAM] = gradient of the mean loss over nrec records (feat[nrec][12],
 * target[nrec] = r, accepted[nrec]); *loss = the mean loss (loss may be NULL).  The
 * summation order is fixed: results are reproducible bit for bit.  Keeps a workspace of
 * per-block partial gradients for each device (grown on demand, synchronising): calls on
 * one device must not overlap.  Errors: HC_EINVAL, HC_ENOMEM, HC_ECUDA. */
int hc_mlp_grad(const float *params, int nrec, const float *feat, const float *target,
                const int32_t *accepted, float kappa, float *grad, float *loss, void *stream);

/* One AdamW step (decoupled weight decay) of the float32 master weights; m1, m2 are the
 * moment buffers (zero before step 1), step counts from 1.  Errors: HC_EINVAL, HC_ECUDA. */
int hc_mlp_adamw(float *params, float *m1, float *m2, const float *grad, int step, float lr,
                 float beta1, float beta2, float eps, float wd, void *stream);

/* out[nrec] = m for each feature record.  Errors: HC_EINVAL, HC_ECUDA. */
int hc_mlp_forward(const float *params, int nrec, const float *feat, float *out, void *stream);

/* Message describing the last failure on the calling host thread ("" if none). */
const char *hc_last_error(void);

/*
 * hc_probe_fp64_peak -- measurement helper, not part of the method: times independent
 * FP64 FMA chains on every SM of the current device and returns, in *gops, the FP64
 * instruction rate in 10^9 instructions per second (one FMA = one instruction).
 * Synchronous.  Errors: HC_ECUDA.
 */
int hc_probe_fp64_peak(double *gops);

/*
 * hc_eval_jac_noalloc -- hc_eval_jac for callers that cannot allocate device memory.
 * The paper has no counterpart: this entry point exists for users of the library.
 *
 * hc_eval_jac allocates its workspace on first use.  A caller whose device memory is
 * owned by its own pool allocator (a framework's caching allocator, a server that
 * reserves a fixed budget at start-up) cannot allow that: the library's cudaMalloc could
 * fail or fragment the pool, and cudaMalloc/cudaFree may synchronise the device inside a
 * latency-critical loop.  This variant calls no allocating routine.  Its workspace is a
 * fixed 32 MiB (33,554,432-byte) array compiled into the library as a device global; a
 * device holds it from the first call on that device (from module load where lazy
 * loading is off) until the process exits.
 *   - A call needing more workspace than that fails with HC_EINVAL before any launch.
 *     The workspace is the power table, (max_exp - 2) * 2 * L * n * npts doubles
 *     (none when every exponent is at most 2): e.g. at most 16,384 points per call for
 *     n = 32, exponents up to 4, DD.  Split larger point sets over several calls.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.  The address is cached per device for the life of the process: a
 *     cudaDeviceReset destroys the array with the context, so after a reset (which ends
 *     every allocation of the process on that device anyway) this entry point must not
 *     be called again on that device.
 *   - Every call uses the same array: calls whose kernels overlap on the GPU (other
 *     streams, other host threads) race on it, so serialise them.  Each call writes the
 *     whole table before reading it, so the previous call's contents do no harm.
 *   - The event-timing helper below must be off (its default): it creates CUDA events.
 * Arguments, layouts, results and other errors are those of hc_eval_jac.
 */
int hc_eval_jac_noalloc(hc_system *sys, int npts, double t, const double *x, double *f,
                        double *J, void *stream);

/*
 * hc_prof_enable / hc_prof_read -- measurement helpers, not part of the method.  While
 * enabled, every launch of the evaluation kernel is bracketed by two CUDA events on the
 * stream it runs on.  hc_prof_read waits for the recorded launches, returns their summed
 * device time in milliseconds and their number, and forgets them.  Host-side state,
 * process-wide; not thread-safe.  Errors: HC_ECUDA.
 */
int hc_prof_enable(int on);
int hc_prof_read(double *ms, int *launches);

#ifdef __cplusplus
}
#endif
#endif /* HC_H */
