/*
 * pgvimp_oracle.h -- plain, slow FP64 CPU oracle of the P-GVIMP hot path
 * (proximal Gaussian variational inference motion planning, arXiv 2411.03416).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the two only meet
 * through the seeded input generators.
 *
 * Conventions: all matrices row-major FP64.  A block-tridiagonal symmetric
 * matrix over N+1 states of dimension n is stored as
 *   diag[i]  = block (i,i),      i = 0..N,   (N+1)*n*n doubles
 *   off[i]   = block (i+1,i),    i = 0..N-1, N*n*n doubles (the lower block;
 *                                            block (i,i+1) is its transpose).
 * Cross covariances follow the same rule: Soff[i] = Sigma_{i+1,i}.
 * The state is x = [q; qdot] with n = 2*nq for every robot model here.
 *
 * Parity status: every function is pinned by the CPU tests.  The hinge/SDF
 * quadrature values, for which the paper prints no numbers, are pinned against
 * independent integrals of the exact SDF of one disk (2-D, E[psi] and its
 * first moment) and one sphere (3-D, E[psi]), besides the affine-SDF special
 * case.  The arm cost is pinned by its planar special case (zero link twists
 * and offsets: the textbook planar-arm formula over an affine SDF), and the
 * twist and offset terms of the DH chain by a closed-form FK of a chain with
 * +pi/2 twists and non-zero offsets written out from the geometry.  The
 * natural-gradient update is pinned by a finite-difference evaluation of the
 * Fisher matrix and the gradient in natural parameters, and by its fixed points.
 */
#ifndef PGVIMP_ORACLE_H
#define PGVIMP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_COST_NONE = 0, ORA_COST_POINT2D = 1, ORA_COST_POINT3D = 2, ORA_COST_ARM = 3, ORA_COST_QUADRATIC = 4 };
enum { ORA_DYN_LINEAR = 0, ORA_DYN_PLANAR_QUAD = 1, ORA_DYN_AFFINE_TEST = 2 };
enum { ORA_RULE_GH = 0, ORA_RULE_DEG3 = 1, ORA_RULE_SMOLYAK = 2 };
enum { ORA_OK = 0, ORA_EINVAL = 1, ORA_ENOTPD = 2, ORA_ENOMEM = 3 };

typedef struct {
  int n, m, N;              /* state dim, noise dim, number of steps (N+1 states) */
  double T;                 /* horizon [s]; dt = T/N */
  const double *A;          /* n*n (LTI) or N*n*n (A_per_step = 1) */
  int A_per_step;
  const double *a;          /* NULL, n, or N*n (a_per_step = 1) */
  int a_per_step;
  const double *B;          /* n*m */
  const double *Qc;         /* m*m */
  const double *mu0, *K0, *muN, *KN;   /* start / goal Gaussians */
  /* collision cost psi_i(x_i) */
  int cost_kind;
  int psi_form;             /* 0: sigma_obs*h^2 (weight), 1: h^2/sigma_obs^2 */
  int factor_set;           /* 0: states 0..N, 1: states 1..N-1 */
  double eps;               /* hinge margin (point robots) / eps_sdf (arm) */
  double sigma_obs;
  double temperature;       /* T-hat; <= 0 means 1 */
  int sdf_nx, sdf_ny, sdf_nz;
  double sdf_origin[3];
  double sdf_cell;
  const float *sdf;         /* index (iz*ny + iy)*nx + ix, node-centred */
  /* arm (cost_kind ARM): nq revolute joints, standard DH rows (a, alpha, d, theta0) */
  int arm_dof;
  const double *dh;         /* arm_dof*4 */
  int n_spheres;
  const int *sphere_link;   /* joint index j in 0..arm_dof-1 */
  const double *sphere_off; /* n_spheres*3, in frame T_{j-1} Rz(theta_j) */
  const double *sphere_r;   /* n_spheres */
  /* quadratic pseudo-cost (tests): psi_i = 1/2 (x-c_i)^T W_i (x-c_i) */
  const double *quad_c;     /* (N+1)*n */
  const double *quad_W;     /* (N+1)*n*n */
  /* nonlinear prior drift for SLR */
  int dyn_kind;
  double dyn_params[4];     /* planar quadrotor: mass, arm length, inertia, gravity */
  const double *dyn_F;      /* affine test drift f(x) = F x + c: n*n */
  const double *dyn_c;      /* n */
} ora_problem;

typedef struct {
  int rule;                 /* ORA_RULE_GH (tensor, gh_p points per dim), ORA_RULE_DEG3, or
                               ORA_RULE_SMOLYAK (sparse grid of level gh_p, Lemma 1) */
  int gh_p;
  double beta_max;          /* first trial step size */
  double kl_eps;            /* KL bound (may be +inf) */
  int max_bisect;
  int iters;                /* proximal iterations (per SLR iteration for SLR plans) */
  int slr_iters;
  int init_kind;            /* 0: Lambda0 = K^-1; 1: Lambda0 = init_scale * I */
  double init_scale;
  const double *replay_beta;/* if non-NULL: step beta_k is given.  The oracle still runs its own
                               search from the current iterate (recorded as beta_own and in the
                               trial records), then takes beta_k whenever Lambda'(beta_k) is
                               positive definite, recording (not enforcing) its KL */
  /* two-phase temperature (the planning experiments of Sec. 7 run a low, then
     a high temperature): from global iteration switch_iter on (> 0), T-hat =
     temperature_high (> 0) in place of the problem's temperature */
  double temperature_high;
  int switch_iter;
  /* the update of each iteration: ORA_UPDATE_PROX (Thm 1, KL proximal term) or ORA_UPDATE_NGD
     (Sec. 3.1(d): natural-gradient step, i.e. the symmetrised KL as the proximal term, taken to
     second order); both with the same step-size search */
  int update;
  /* optional record of every trial of the own step-size search (NULL: none); *trials_n counts
     the records written, at most trials_cap */
  struct ora_trial_rec *trials_out;
  int trials_cap;
  int *trials_n;
} ora_options;

enum { ORA_UPDATE_PROX = 0, ORA_UPDATE_NGD = 1 };

typedef struct {
  double beta, kl, kl_margin, prior_cost, collision_cost, entropy;
  int trials, accepted;
  double beta_own;          /* the step the oracle's own search chose (= beta unless replayed) */
  double pd_margin;         /* min over the own search's trials of |smallest relative pivot| */
  int replayed;             /* 1 if beta is a replayed step that differs from beta_own */
  int pad;
} ora_iter_log;

/* One trial of the step-size search (App. C). */
typedef struct ora_trial_rec {
  int iter;                 /* global iteration index */
  int pd;                   /* Lambda'(beta) positive definite */
  int feasible;             /* pd and KL <= eps */
  int pad;
  double beta;
  double kl;                /* +inf when not pd */
  double rel_pivot;         /* smallest pivot of the block elimination of Lambda'(beta) divided by
                               the diagonal entry it came from; <= 0 where the elimination failed */
} ora_trial_rec;

/* ---- dense helpers (exposed for the pins) ---- */
int ora_expm(int d, const double *M, double *E);
int ora_gh_rule(int p, double *nodes, double *weights);
int ora_rule_size(int n, int rule, int p);
int ora_rule(int n, int rule, int p, double *xi, double *W);

/* ---- prior (Alg. 1, first two lines) ---- */
int ora_prior(const ora_problem *pb, const double *A_ltv, const double *a_ltv,
              double *Kd, double *Ko, double *b, double *Phi, double *Q, double *u);
int ora_prior_mean(const ora_problem *pb, const double *Kd, const double *Ko, const double *b, double *mubar);
int ora_init_mean(const ora_problem *pb, double *mu);

/* ---- marginals by Gaussian belief propagation (Sec. 5.1) ---- */
int ora_marginals(int n, int N, const double *Ld, const double *Lo, double *Sd, double *So, double *logdet);
/* as ora_marginals, also returning the smallest relative pivot of the forward pass (rel_pivot may be
   NULL); on ORA_ENOTPD rel_pivot holds the failing pivot (<= 0) */
int ora_marginals_pivot(int n, int N, const double *Ld, const double *Lo, double *Sd, double *So,
                        double *logdet, double *rel_pivot);
int ora_block_solve(int n, int N, const double *Md, const double *Mo, const double *r, double *x);

/* ---- factor expectations (Sec. 4.2-4.3) ---- */
double ora_sdf(const ora_problem *pb, const double *pos);
int ora_arm_fk(const ora_problem *pb, const double *q, double *centres);
double ora_psi(const ora_problem *pb, int i, const double *x);
int ora_quad_moments(const ora_problem *pb, const ora_options *op, int i, const double *mu_i,
                     const double *Sig_ii, double *S0, double *S1, double *S2);
int ora_gradients(int n, const double *Sig_ii, double S0, const double *S1, const double *S2,
                  double *g, double *G);

/* ---- KL-proximal update (Thm 1) and step-size search (App. C) ---- */
int ora_trial(const ora_problem *pb, double beta, const double *Kd, const double *Ko, const double *b,
              const double *mu, const double *Ld, const double *Lo, double logdet_k,
              const double *g, const double *G,
              double *mu_new, double *Ld_new, double *Lo_new, double *Sd_new, double *So_new,
              double *logdet_new, double *kl);
/* the trial of either update (ORA_UPDATE_PROX: Thm 1; ORA_UPDATE_NGD: Sec. 3.1(d)), with the
   smallest relative pivot of Lambda'(beta) (may be NULL) */
int ora_trial_ex(const ora_problem *pb, int update, double beta, const double *Kd, const double *Ko,
                 const double *b, const double *mu, const double *Ld, const double *Lo, double logdet_k,
                 const double *g, const double *G,
                 double *mu_new, double *Ld_new, double *Lo_new, double *Sd_new, double *So_new,
                 double *logdet_new, double *kl, double *rel_pivot);
int ora_step(const ora_problem *pb, const ora_options *op, int k,
             const double *Kd, const double *Ko, const double *b, const double *mubar,
             double *mu, double *Ld, double *Lo, double *Sd, double *So, double *logdet,
             ora_iter_log *out_log);

/* ---- drivers (Alg. 1, Alg. 2) ---- */
int ora_plan(const ora_problem *pb, const ora_options *op, int init, double *mu, double *Ld,
             double *Lo, double *Sd, double *So, ora_iter_log *logs);
int ora_drift(const ora_problem *pb, const double *x, double *f);
int ora_slr(const ora_problem *pb, const ora_options *op, const double *xbar, const double *Sbar,
            double *A_out, double *a_out);
int ora_plan_slr(const ora_problem *pb, const ora_options *op, double *mu, double *Ld, double *Lo,
                 double *Sd, double *So, ora_iter_log *logs, double *slr_norms);

#ifdef __cplusplus
}
#endif
#endif
