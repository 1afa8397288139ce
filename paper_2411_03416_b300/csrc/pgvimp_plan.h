// pgvimp_plan.h -- per-plan device descriptor shared by the host API and the
// kernels of the CUDA library (internal; not part of the C ABI).
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/pgvimp.h"

namespace pgv {

constexpr int kMaxN = 16;        // largest state dimension
constexpr int kMaxDof = 8;       // largest arm chain
constexpr int kMaxSpheres = 64;
constexpr int kMaxGH = 10;       // largest points-per-dimension of the GH rule
constexpr int kScal = 24;        // per-plan scalar slots
constexpr int kCrMaxThreads = 256; // largest thread block of the block (latency) form
constexpr int kLaneThreads = 16;   // plan_threads value of the lane form (sixteen lanes per plan, n = 4)

// Per-plan scalar slots (doubles).
enum ScalSlot {
  S_LOGDET = 0,       // log det Lambda_k
  S_T_LOGDET = 1,     // log det Lambda' of the last trial
  S_T_KL = 2,         // KL of the last trial
  S_T_PD = 3,         // 1 if the last trial's Lambda' was positive definite
  S_COLL = 4,         // sum_i E[psi_i] at the last quadrature
  S_K = 5,            // global proximal iteration counter
  S_KIN = 6,          // iteration counter within the current linearisation
  S_J = 7,            // SLR linearisation counter
  S_INIT = 8,         // 1 once the plan has been initialised
  S_CUR = 9,          // buffer set holding (mu, Sigma) of the current iterate
  S_PRIOR = 10,       // prior cost of the current iterate
  S_T_PRIOR = 11,     // prior cost of the last trial's iterate
  S_STATUS = 12,      // 0 ok; 1 prior not PD; 2 marginals of Lambda_k not PD; 3 quadrature factor not PD
  S_T_DELTA = 13,     // delta^T Lambda_k delta of the last trial
  S_T_TRACE = 14,     // tr((Lambda_k - Lambda') Sigma') of the last trial
  S_T_BEST = 15,      // best-feasible buffer set during a search
  S_NSETS = 16,
  S_FMT = 17,          // double-float storage: 1 while the result buffers hold FP64
  S_THIGH = 18         // 1 once K^-1 and b are divided by the high temperature
};

// Sets the calling thread's error text returned by pgvimp_last_error(NULL).
void set_thread_error(const char* msg);
inline void set_thread_error(const std::string& msg) { set_thread_error(msg.c_str()); }

struct PlanDesc;
struct Launch {
  const PlanDesc* descs;
  int count;
  cudaStream_t stream;
};

struct PlanDesc {
  // sizes and options
  int n, m, N, nq, dc;
  double T, dt;
  int rule, gh_p, max_bisect, iters, slr_iters, init_kind;
  int update;                  // pgvimp_update: Thm 1 step or natural-gradient step
  double beta_max, kl_eps, init_scale;
  // cost
  int cost_kind, psi_form, factor_set;
  double eps, sigma_obs, inv_temp;
  double inv_temp_high;        // 1 / high temperature from iteration switch_iter on (0: one phase)
  int switch_iter;
  int nx, ny, nz;
  double sdf_origin[3];
  double cell, inv_cell;
  const float* sdf;
  int arm_dof, n_spheres;
  const double* dh;            // arm_dof*4
  const double* sphere_off;    // n_spheres*3, grouped by link
  const double* sphere_r;      // n_spheres
  int sphere_begin[kMaxDof + 1];
  // Gauss-Hermite tables: nodes / weights of the p-point rule at [p * kMaxGH + j]
  const double* gh_x;
  const double* gh_w;
  // Smolyak rule tables (rule SMOLYAK): the collision rule over the dc cost
  // coordinates, rows (xi_0..xi_{dc-1}, weight at level k, weight at level
  // k-1), and for SLR plans the rule over all n dimensions, rows (xi, weight)
  const double* sg;
  const double* sgs;
  int sg_rows, sgs_rows;
  // prior inputs
  int dyn_kind;
  double dyn_params[4];
  const double *A, *a;
  int A_per_step, a_per_step;
  const double *B, *Qc, *mu0, *K0, *muN, *KN;
  // state (device arena)
  double *Kd, *Ko, *b, *mubar;
  double *Ld, *Lo;
  double *mu[3], *Sd[3], *So[3];   // three buffer sets: current / best / trial rotate
  double *g, *G;
  double *Altv, *altv, *xbar;
  double *scr;                     // per-step factorisation scratch
  double *scal;                    // kScal doubles
  double *slr_norms;               // slr_iters doubles
  pgvimp_step_info* log;
  int log_cap;
};

}  // namespace pgv
