/*
 * pgvimp.h -- C ABI of the B300 (sm_103a) implementation of P-GVIMP, the
 * parallel proximal Gaussian variational inference motion planner of
 * "Efficient Iterative Proximal Variational Inference Motion Planning"
 * (arXiv 2411.03416; referred to below by section, equation and algorithm).
 *
 * The library solves, for one or many planning problems at once, the
 * discretised variational problem of Sec. 2.2: a Gaussian trajectory
 * distribution q = N(mu, Lambda^-1) over states x_0..x_N of an LTV SDE
 *   dX = (A_t X + a_t) dt + B dW,  E[dW dW^T] = Qc dt        (Sec. 2.2)
 * with soft start / goal Gaussians, a collision cost on a signed-distance
 * field (Sec. 4.1), optimised by the KL-proximal iteration of Thm 1 with the
 * KL-bounded step-size search of App. C (Alg. 1), or, for a nonlinear prior
 * drift, by the SLR outer loop of Alg. 2 (Sec. 6.2).  Every step of that path
 * runs in this library's CUDA kernels; there is no CPU fallback.
 *
 * Entry points: single plans (pgvimp_create / step / plan / get / destroy),
 * batches of independent plans (pgvimp_batch_*), single rows of the path for
 * inspection (pgvimp_batch_phase), a continuous-batching server
 * (pgvimp_server_*), and an allocation-free marginals call.  Each plan runs
 * in one of three execution forms chosen by pgvimp_options.plan_threads: one
 * GPU thread per plan (throughput), sixteen lanes per plan for n = 4
 * (throughput, one block element per lane), or one thread block per plan with
 * the block recursions by cyclic reduction over time (latency; one warp per
 * elimination for n >= 6).
 *
 * General rules for every entry point:
 *  - all functions are extern "C", never throw, never abort and return a
 *    pgvimp_status; on failure pgvimp_last_error() gives a one-line reason;
 *  - host pointers are read during the call only (inputs are deep-copied);
 *    the caller keeps ownership of every buffer it passes;
 *  - `stream` arguments are cudaStream_t handles passed as void*; NULL is the
 *    legacy default stream;
 *  - matrices are row-major FP64 unless stated; block-tridiagonal symmetric
 *    matrices over the N+1 states are stored as diagonal blocks (N+1) x n x n
 *    and lower off-diagonal blocks (N) x n x n (block (i+1, i)); block (i, i+1)
 *    is the transpose.  Cross covariances use the same rule.
 */
#ifndef PGVIMP_H
#define PGVIMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PGVIMP_OK = 0,
  PGVIMP_EINVAL = 1,      /* bad argument, size or option */
  PGVIMP_ENOMEM = 2,      /* device or pinned host memory exhausted / arena too small */
  PGVIMP_ENOTPD = 3,      /* an input covariance (K0, KN, Qc) or the prior is not positive definite */
  PGVIMP_ECUDA = 4,       /* a CUDA runtime call failed */
  PGVIMP_ETIMEOUT = 5,    /* a bounded wait expired */
  PGVIMP_EBUSY = 6,       /* the server's admission queue is full */
  PGVIMP_ENOTFINITE = 7,  /* an input holds NaN or Inf */
  PGVIMP_ENOTREADY = 8    /* a polled request has not finished yet */
} pgvimp_status;

/* Collision cost at a state (Sec. 4.1, the collision factors psi_i). */
typedef enum {
  PGVIMP_COST_NONE = 0,    /* psi = 0 (the GP prior alone) */
  PGVIMP_COST_POINT2D = 1, /* h = max(0, eps - sdf(x_0, x_1)), 2-D bilinear SDF */
  PGVIMP_COST_POINT3D = 2, /* h = max(0, eps - sdf(x_0, x_1, x_2)), 3-D trilinear SDF */
  PGVIMP_COST_ARM = 3      /* sum over body spheres of the hinge at eps + r_s, revolute chain FK */
} pgvimp_cost_kind;

/* Prior drift (Sec. 2.2 for LINEAR; Sec. 6 / eq. planar_quad for SLR). */
typedef enum {
  PGVIMP_DYN_LINEAR = 0,       /* A_t, a_t given */
  PGVIMP_DYN_PLANAR_QUAD = 1   /* f_0 of the planar quadrotor with u = 0, linearised by SLR (Alg. 2) */
} pgvimp_dyn_kind;

typedef enum { PGVIMP_RULE_GH = 0, PGVIMP_RULE_DEG3 = 1, PGVIMP_RULE_SMOLYAK = 2 } pgvimp_rule;

/* The update taken at each iteration (both with the KL-bounded step-size
 * search of App. C).  PROX: the KL-proximal step of Thm 1 (eq.
 * mu_Sigma_update).  NGD: the natural-gradient step of Sec. 3.1(d),
 * delta theta = beta G(theta)^-1 grad L with the Fisher matrix G, taken in the
 * natural parameters (Lambda mu, -Lambda/2):
 *   Lambda' = (1 - beta) Lambda_k + beta (K^-1 + 2 grad_Sigma psi_d),
 *   Lambda' mu' = (1 - beta) Lambda_k mu_k + beta (K^-1 mu_bar - grad_mu psi_d
 *                 + 2 grad_Sigma psi_d mu_k);
 * it needs beta_max <= 1. */
typedef enum { PGVIMP_UPDATE_PROX = 0, PGVIMP_UPDATE_NGD = 1 } pgvimp_update;

/* Arithmetic of the path.  PLAIN_FP64: everything in FP64.  MIXED: the
 * quadrature, SDF and moment arithmetic in FP32 (FP32 accumulation); the
 * marginal recovery, the update and the KL / step-size search in FP64.
 * MIXED_DF: as MIXED, but the recursions run in double-float arithmetic
 * (pairs of FP32 values, ~48-bit significand) on the FP32 pipe, which on B300
 * issues at 64x the FP64 rate; results are returned in FP64.  Its errors
 * follow its ~2^-48 unit roundoff: on precision matrices conditioned at
 * 6e11 to 4e12 (dense 750-step horizons through clutter) the marginal
 * covariances after one iteration were 1e-3 to 6e-3 from the FP64 oracle,
 * against 1e-4 with MIXED, so MIXED is the form whose stated error bounds
 * hold on every input.  The single-row phases (pgvimp_batch_phase other
 * than PRIOR) need PLAIN_FP64 or MIXED. */
typedef enum { PGVIMP_PREC_PLAIN_FP64 = 0, PGVIMP_PREC_MIXED = 1, PGVIMP_PREC_MIXED_DF = 2 } pgvimp_precision;

/* One planning problem.  All pointers are host pointers, row-major FP64
 * unless stated.  The state is x = [q; qdot], n = 2*nq. */
typedef struct {
  int n;            /* state dimension: 4, 6 or 14 (kernels are compiled per size) */
  int m;            /* noise dimension, 1..16 */
  int N;            /* number of steps; N+1 states on t_i = i*T/N; N >= 1 */
  double T;         /* horizon [s] */
  const double *A;  /* LINEAR: n*n (A_per_step = 0) or N*n*n; ignored for SLR models */
  int A_per_step;
  const double *a;  /* NULL (zero), n, or N*n (a_per_step = 1) */
  int a_per_step;
  const double *B;  /* n*m */
  const double *Qc; /* m*m, symmetric positive definite */
  const double *mu0, *K0;   /* start Gaussian: n, n*n */
  const double *muN, *KN;   /* goal Gaussian: n, n*n */
  int cost_kind;    /* pgvimp_cost_kind */
  int psi_form;     /* 0: psi = sigma_obs*h^2; 1: psi = h^2/sigma_obs^2 */
  int factor_set;   /* 0: collision factors on states 0..N; 1: on 1..N-1 */
  double eps;       /* hinge margin (point robots) or eps_sdf (arm) [m] */
  double sigma_obs; /* obstacle weight, > 0 */
  double temperature; /* T-hat > 0 (<= 0 means 1); scales prior and cost by 1/T-hat */
  int sdf_nx, sdf_ny, sdf_nz;   /* grid nodes; nz <= 1 for a 2-D map; each >= 2 when used */
  double sdf_origin[3];         /* position of node (0,0,0) [m] */
  double sdf_cell;              /* node spacing [m] */
  const float *sdf;             /* FP32, index (iz*ny + iy)*nx + ix */
  int arm_dof;                  /* ARM: revolute joints (= nq) */
  const double *arm_dh;         /* ARM: arm_dof*4 standard DH rows (a, alpha, d, theta0) */
  int n_spheres;                /* ARM: body spheres, <= 64 */
  const int *sphere_link;       /* ARM: joint index of each sphere */
  const double *sphere_off;     /* ARM: n_spheres*3 offsets in the frame T_{j-1} Rz(theta_j) */
  const double *sphere_r;       /* ARM: radii */
  int dyn_kind;                 /* pgvimp_dyn_kind */
  double dyn_params[4];         /* PLANAR_QUAD: mass, arm length, inertia, gravity */
} pgvimp_problem;

typedef struct {
  int rule;         /* pgvimp_rule: GH tensor rule (gh_p points per dim), degree-3 (2n+1 points), or
                       Smolyak sparse grid of level gh_p (Lemma 1: 1-D GH rules with 1..gh_p points,
                       exact for total degree 2 gh_p - 1) */
  int gh_p;         /* 2..10 */
  double beta_max;  /* first trial step size (App. C), > 0 */
  double kl_eps;    /* KL bound epsilon (may be +inf) */
  int max_bisect;   /* halvings of [0, beta_max] after an infeasible first trial, 0..60 */
  int iters;        /* proximal iterations (per SLR linearisation) */
  int slr_iters;    /* SLR linearisations (Alg. 2); ignored for LINEAR */
  int init_kind;    /* 0: Lambda_0 = K^-1; 1: Lambda_0 = init_scale * I */
  double init_scale;
  int plan_threads; /* execution form (same for every plan of a batch; not part of the method):
                       1: one GPU thread per plan, sequential sweeps over time (thread form);
                       16: sixteen lanes per plan, one element of each n x n block per lane,
                       sequential sweeps over time (lane form; n = 4 only);
                       0: the default throughput form: the lane form for n = 4 with MIXED_DF
                       precision, the thread form otherwise;
                       32..256, a multiple of 32: one thread block of that size per plan, the block
                       recursions by cyclic reduction over time (latency form), in any precision. */
  double temperature_high; /* two-phase temperature (the low/high T-hat schedule of the planning
                              experiments, Sec. 7): from global iteration switch_iter on (> 0), K^-1, b
                              and the cost are divided by temperature_high (> 0) instead of the
                              problem's temperature; 0 or switch_iter = 0: one phase */
  int switch_iter;
  int update;       /* pgvimp_update (0: Thm 1) */
} pgvimp_options;

/* Per-iteration record.  Costs are those of the iterate the gradients were
 * taken at: prior = 1/2 [tr(K^-1 Sigma) + (mu - mu_bar)^T K^-1 (mu - mu_bar)],
 * collision = sum_i E[psi_i], entropy = 1/2 log det(2 pi e Sigma). */
typedef struct {
  double beta;        /* accepted step (0: no move) */
  double kl;          /* KL(q_{k+1} || q_k) of the accepted step */
  double kl_margin;   /* min over trials of |KL - eps| / eps (tie detector) */
  double prior_cost, collision_cost, entropy;
  int trials;         /* trial steps evaluated */
  int iter;           /* global iteration index */
} pgvimp_step_info;

/* ------------------------------------------------------------------ batches
 * A batch holds `count` problems of one state dimension, one cost kind and
 * one precision, each with its own N, map and options, resident in device
 * memory.  One call of pgvimp_batch_run advances every plan; each GPU thread
 * owns one plan.  A batch is used by one host thread at a time. */
typedef struct pgvimp_batch pgvimp_batch;

/* Device bytes a batch needs (inputs, state, scratch, logs).  The layout
 * holds, per plan, the prior (K^-1 blocks, b, mu_bar; Alg. 1, first two
 * lines), the iterate (mu, Lambda blocks) and its marginals (Sec. 5.1), the
 * gradients g, G (Sec. 4.2), trial buffers of the step-size search (App. C)
 * and, for SLR models, the linearisation A_i, a_i (Sec. 6.2).  EINVAL as
 * pgvimp_batch_create. */
pgvimp_status pgvimp_batch_arena_bytes(int count, const pgvimp_problem *problems,
                                       const pgvimp_options *options, int precision, size_t *bytes);

/* Validates and deep-copies the problems into pinned host staging and lays
 * them out in a device arena: `arena` (caller-owned device memory of
 * `arena_bytes` >= pgvimp_batch_arena_bytes, e.g. from PyTorch; 256-byte
 * aligned) or, if NULL, memory the batch allocates itself.  Validation:
 * dimensions and options in range (EINVAL), finite inputs (ENOTFINITE),
 * K0, KN, Qc symmetric positive definite (ENOTPD). */
pgvimp_status pgvimp_batch_create(int count, const pgvimp_problem *problems, const pgvimp_options *options,
                                  int precision, void *arena, size_t arena_bytes, pgvimp_batch **out);

/* Host-to-device copy of every problem's inputs (from the pinned staging). */
pgvimp_status pgvimp_batch_upload(pgvimp_batch *b, void *stream);

/* Marks every plan as not started: the next run begins with the prior build
 * (Alg. 1, first two lines) and the initial iterate. */
pgvimp_status pgvimp_batch_reset(pgvimp_batch *b, void *stream);

/* Advances every plan by `iters` proximal iterations (<= 0: the whole plan,
 * options.iters, times options.slr_iters for SLR models): the loop of Alg. 1
 * -- factor expectations (Sec. 4.3, 5.2), gradients (eq. gradients_psid),
 * the update of Thm 1 (or NGD, Sec. 3.1(d)) with the KL-bounded step-size
 * search (App. C), marginals of the new precision (Sec. 5.1).  A plan that
 * has not started is first initialised (prior and initial iterate, the set-up of Alg. 1).  SLR models
 * relinearise (Sec. 6.2, Alg. 2) at the start of each outer iteration.
 * Asynchronous on `stream`; a plan that fails (prior or marginals not PD)
 * records its status and stops, the others continue. */
pgvimp_status pgvimp_batch_run(pgvimp_batch *b, int iters, void *stream);

/* Device-to-host copy of the results (means, marginal covariances, precision
 * blocks, logs, status) into pinned staging. */
pgvimp_status pgvimp_batch_download(pgvimp_batch *b, void *stream);

/* Device-to-host copy of the result section only: means, marginal
 * covariances Sigma_ii, logs and status (pgvimp_batch_result then returns
 * those; cross covariances and precision blocks are not refreshed). */
pgvimp_status pgvimp_batch_download_results(pgvimp_batch *b, void *stream);

/* Reads plan `index` from the staging filled by the last download (call
 * after synchronising its stream).  Any output pointer may be NULL.
 * mu: (N+1)*n; Sd/Ld: (N+1)*n*n; So/Lo: N*n*n; logs: up to max_logs records. */
pgvimp_status pgvimp_batch_result(const pgvimp_batch *b, int index, double *mu, double *Sd, double *So,
                                  double *Ld, double *Lo, pgvimp_step_info *logs, int max_logs, int *n_logs);

/* Bytes moved by one upload / one full download / one results-only download. */
pgvimp_status pgvimp_batch_io_bytes(const pgvimp_batch *b, size_t *h2d, size_t *d2h, size_t *d2h_results);
pgvimp_status pgvimp_batch_destroy(pgvimp_batch *b);

/* -------------------------------------------------- single steps of the path
 * Each runs one row of the hot path for every plan of a batch, on the same
 * device code the fused run uses, so that each row can be checked on its own.
 * Buffers are read and written with pgvimp_batch_read / pgvimp_batch_write. */
typedef enum {
  PGVIMP_PHASE_PRIOR = 0,     /* the set-up of Alg. 1: Phi_i, Q_i (Van Loan), K^-1, b; initial mu, Lambda */
  PGVIMP_PHASE_MARGINALS = 1, /* Sec. 5.1: Sigma_ii, Sigma_{i+1,i}, log det of the current Lambda */
  PGVIMP_PHASE_QUAD = 2,      /* Sec. 4.1-4.3: E[psi_i] and the gradients g_i, G_i at (mu, Sigma_ii) */
  PGVIMP_PHASE_TRIAL = 3,     /* Thm 1 at step `arg`: mu', Sigma' blocks, log det, KL, feasibility */
  PGVIMP_PHASE_SLR = 4        /* Sec. 6.2: A_i, a_i from the nominal (mu, Sigma_ii) */
} pgvimp_phase;
pgvimp_status pgvimp_batch_phase(pgvimp_batch *b, int phase, double arg, void *stream);

typedef enum {
  PGVIMP_BUF_MU = 0, PGVIMP_BUF_LD = 1, PGVIMP_BUF_LO = 2, PGVIMP_BUF_SD = 3, PGVIMP_BUF_SO = 4,
  PGVIMP_BUF_KD = 5, PGVIMP_BUF_KO = 6, PGVIMP_BUF_B = 7, PGVIMP_BUF_G1 = 8 /* g: (N+1)*n */,
  PGVIMP_BUF_G2 = 9 /* G: (N+1)*n*n */, PGVIMP_BUF_TMU = 10 /* trial mu' */, PGVIMP_BUF_TSD = 11,
  PGVIMP_BUF_TSO = 12, PGVIMP_BUF_ALTV = 13 /* N*n*n */, PGVIMP_BUF_ALTVA = 14 /* N*n */,
  PGVIMP_BUF_SCAL = 15 /* 8 doubles: logdet, trial logdet, trial kl, trial pd, collision, k, j, status */
} pgvimp_buffer;
/* Synchronous copies between a plan's device buffer and host memory;
 * `count` doubles must equal the buffer's size (EINVAL otherwise). */
pgvimp_status pgvimp_batch_read(const pgvimp_batch *b, int index, int buffer, double *host, size_t count);
pgvimp_status pgvimp_batch_write(pgvimp_batch *b, int index, int buffer, const double *host, size_t count);

/* ------------------------------------------------------- single-plan context
 * The calls of Alg. 1 / Alg. 2 for one problem: a batch of one, on the
 * library's own stream, with its own device memory. */
typedef struct pgvimp_ctx pgvimp_ctx;
/* Sets up one problem in the form of Sec. 2.2: the LTV SDE (A_t, a_t, B, Qc)
 * discretised on t_i = i T/N, the start and goal Gaussians, the collision cost
 * on an SDF (Sec. 4.1) and the method's options; deep-copies the inputs and
 * uploads them.  Validation and errors as pgvimp_batch_create; ENOMEM if the
 * device or pinned memory runs out. */
pgvimp_status pgvimp_create(const pgvimp_problem *problem, const pgvimp_options *options, int precision,
                            pgvimp_ctx **out);
/* One iteration of Alg. 1: the factor expectations and gradients at the
 * current iterate, the update of Thm 1 (eq. mu_Sigma_update; NGD with
 * options.update) at the largest step the KL bound of App. C admits, and the
 * marginals of the new precision.  For SLR models, the relinearisation of
 * Sec. 6.2 precedes the first iteration of each outer step of Alg. 2.  Blocks
 * until done; `info` (may be NULL) receives the iteration's record. */
pgvimp_status pgvimp_step(pgvimp_ctx *ctx, pgvimp_step_info *info);
/* `iters` iterations (<= 0: the whole plan: Alg. 1 for options.iters
 * iterations, or Alg. 2 for options.slr_iters linearisations of
 * options.iters iterations each).  Blocks until done. */
pgvimp_status pgvimp_plan(pgvimp_ctx *ctx, int iters);
/* The current Gaussian N(mu, Lambda^-1): mu ((N+1)*n), the marginal
 * covariances Sigma_ii of Sec. 5.1 ((N+1)*n*n) and the precision blocks
 * Lam_diag ((N+1)*n*n) / Lam_off (N*n*n), all FP64 into caller-owned host
 * buffers.  Any pointer may be NULL. */
pgvimp_status pgvimp_get(pgvimp_ctx *ctx, double *mu, double *Sigma, double *Lam_diag, double *Lam_off);
/* Frees the context and its device memory.  NULL-safe. */
pgvimp_status pgvimp_destroy(pgvimp_ctx *ctx);

/* Last error text of a context (or of the calling thread if ctx is NULL). */
const char *pgvimp_last_error(const void *ctx);

/* ------------------------------------------------------------------ serving
 * A server plans requests as they arrive (continuous batching).  Requests of
 * the same state dimension and dynamics kind that wait at the same time are
 * packed into one batch; each batch runs the whole plan (Alg. 1, or Alg. 2
 * for SLR models) on one of `max_inflight` streams, so batches admitted while
 * others run overlap on the GPU.  Each batch's launch sequence (copy in,
 * prior, iterations, copy out, completion) is captured into a CUDA graph and
 * launched as one; a stream's executable graph is updated in place for the
 * next batch of the same shape.  A batch is admitted when a stream is free
 * and its device arena and pinned staging fit the server's pools, which are
 * allocated once at creation; a request waits at most `batch_window_ms` for
 * others to share its launch.  All server functions are thread-safe.
 * Streams beyond the device's hardware work queues share queues and their
 * kernels serialise: run the process with CUDA_DEVICE_MAX_CONNECTIONS >=
 * max_inflight (at most 32) set before the CUDA context is created. */
typedef struct pgvimp_server pgvimp_server;
typedef struct {
  size_t hbm_budget_bytes;   /* device pool for admitted batches (>= 1 MiB) */
  size_t host_staging_bytes; /* pinned host pool (0: min(hbm_budget_bytes, 4 GiB)) */
  int precision;             /* pgvimp_precision of every served plan */
  int plan_threads;          /* execution form of every served plan (pgvimp_options.plan_threads), or -1:
                                each request's own options.plan_threads (e.g. from an autotuner) */
  int max_inflight;          /* batches on the device at once, 1..64 */
  int max_batch;             /* plans per batch, >= 1 */
  double batch_window_ms;    /* longest wait of a queued request for batch company, >= 0 */
} pgvimp_server_config;
typedef struct {
  int status;                /* pgvimp_status of the plan */
  int n, N, n_logs;          /* sizes and number of iteration records */
  int batch_size;            /* plans in the batch that carried the request */
  double submit_ms, start_ms, done_ms;   /* server clock: submitted, launched, result on the host */
  pgvimp_step_info last;     /* last iteration record */
} pgvimp_request_info;
typedef struct {
  int queued, inflight;      /* requests waiting, batches on the device */
  uint64_t batches, plans;   /* launched so far */
  size_t dev_used, host_used;
  double now_ms;             /* server clock */
  double host_launch_ms;     /* scheduler time spent creating and queueing batches */
  double host_collect_ms;    /* scheduler time spent copying results out */
  uint64_t graph_launches;   /* batches launched as one captured CUDA graph */
  uint64_t graph_instantiations;   /* executable graphs built (the rest were updated in place) */
} pgvimp_server_stats_t;

/* Creates the pools, streams and the scheduler thread on the current device.
 * EINVAL for a bad config, ENOMEM if a pool cannot be allocated. */
pgvimp_status pgvimp_server_create(const pgvimp_server_config *cfg, pgvimp_server **out);
/* Validates and deep-copies one request (the caller may free its arrays on
 * return) and queues it.  options.plan_threads is replaced by the server's
 * unless the server was created with plan_threads = -1.
 * ENOMEM if the request alone exceeds a pool; validation as pgvimp_batch_create. */
pgvimp_status pgvimp_submit(pgvimp_server *s, const pgvimp_problem *problem, const pgvimp_options *options,
                            uint64_t *request_id);
/* Waits up to timeout_ms (< 0: no limit, 0: no wait) for a request; on
 * completion copies mu ((N+1) n) and Sigma ((N+1) n n; either may be NULL),
 * fills info (may be NULL), forgets the request and returns the plan's status.
 * ENOTREADY if it has not finished (the request stays queued). */
pgvimp_status pgvimp_poll(pgvimp_server *s, uint64_t request_id, int timeout_ms, double *mu, double *Sigma,
                          pgvimp_request_info *info);
pgvimp_status pgvimp_server_stats(pgvimp_server *s, pgvimp_server_stats_t *out);
/* Waits for the batches on the device, drops queued requests, frees everything. NULL-safe. */
pgvimp_status pgvimp_server_destroy(pgvimp_server *s);

/* ----------------------------------------------- allocation-free marginals
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory -- code running while its stream is captured
 * into a CUDA graph (cudaMalloc is not capturable and may synchronise the
 * device), runtimes that give a component a fixed memory budget, hosts that
 * own every device byte through their own pool.  It computes the block
 * marginals of a block-tridiagonal SPD precision like PGVIMP_PHASE_MARGINALS
 * (same elimination and selected-inverse sweeps, FP64), but the per-state
 * scratch lives in a fixed device array of 4 MiB compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   n: 4, 6 or 14; N >= 1 with (N+1) * (n(n+1)/2 rounded up to even + n*n)
 *      * 8 bytes <= 4 MiB (n = 4: N <= 20,163; n = 6: N <= 9,038; n = 14: N <= 1,735);
 *      larger sizes return PGVIMP_EINVAL;
 *   Ld, Lo: device input blocks ((N+1) n*n, N n*n); Sd, So: device outputs
 *      (Sigma_ii, Sigma_{i+1,i}); the four 16-byte aligned; logdet: device,
 *      one double (NaN when the precision is not positive definite, in which
 *      case Sd / So are not written).  The caller owns all five buffers.
 * The call allocates nothing and returns after queueing one kernel on
 * `stream`.  Its first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  All
 * calls share the array: calls that overlap on the GPU race on it, so the
 * caller serialises them (one stream, or events).  Errors: PGVIMP_EINVAL for
 * bad sizes or pointers, PGVIMP_ECUDA for a failed launch; the text is
 * available from pgvimp_last_error(NULL). */
pgvimp_status pgvimp_marginals_noalloc(int n, int N, const double *Ld, const double *Lo, double *Sd, double *So,
                                       double *logdet, void *stream);

/* Library build / device information: writes a short text (e.g. "sm_103a"). */
pgvimp_status pgvimp_version(char *buf, size_t len);

/* sizeof of the ABI structs as compiled into the library, so that bindings
 * can check their marshalling: pgvimp_problem, pgvimp_options,
 * pgvimp_step_info.  Any pointer may be NULL. */
pgvimp_status pgvimp_abi_sizes(size_t *problem, size_t *options, size_t *step_info);

#ifdef __cplusplus
}
#endif
#endif /* PGVIMP_H */
