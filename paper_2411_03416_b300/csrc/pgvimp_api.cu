// pgvimp_api.cu -- host side of the C ABI declared in include/pgvimp.h:
// validation, device arena layout, pinned staging, launch orchestration of
// Alg. 1 / Alg. 2, and the single-plan context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "pgvimp_plan.h"

#include "pgvimp_launch.h"
#include "pgvimp_internal.h"

namespace pgv {
// Dispatch of a phase to the kernels of state dimension n and precision.
// `tpb`: threads per plan of the block form (0: not the block form); `lane`:
// the lane form of the fused iterations (n = 4, sixteen lanes per plan).
static cudaError_t launch_phase(int n, const Launch& L, int phase, int arg_i, double arg_d, int precision, int tpb,
                                bool lane) {
  constexpr int PRIOR = 100, INIT = 101, ITER = 102, SLR = 103, RELIN = 104, FIN = 106, WORKING = 107;
  const bool rows = (phase == PGVIMP_PHASE_MARGINALS || phase == PGVIMP_PHASE_QUAD || phase == PGVIMP_PHASE_TRIAL);
  const bool df = (precision == PGVIMP_PREC_MIXED_DF);
  const int qt32 = (precision != PGVIMP_PREC_PLAIN_FP64);
  if (lane && n == 4 && phase == ITER) {
    if (df) return launch_iter_lane<float, df64>(L, arg_i);
    return qt32 ? launch_iter_lane<float, double>(L, arg_i) : launch_iter_lane<double, double>(L, arg_i);
  }
  switch (n) {
#define PGV_CASE(N_)                                                                                      \
  case N_:                                                                                                \
    if (tpb) {                                                                                            \
      if (phase == ITER) {                                                                                \
        if (df) return launch_iter_cta<N_, float, df64>(L, arg_i, tpb);                                   \
        return qt32 ? launch_iter_cta<N_, float, double>(L, arg_i, tpb)                                   \
                    : launch_iter_cta<N_, double, double>(L, arg_i, tpb);                                 \
      }                                                                                                   \
      if (phase == INIT || phase == SLR || phase == PRIOR || phase == RELIN || phase == FIN ||            \
          phase == WORKING)                                                                               \
        return df ? launch_aux_cta<N_, df64>(L, phase, arg_i, qt32, tpb)                                  \
                  : launch_aux_cta<N_, double>(L, phase, arg_i, qt32, tpb);                               \
    }                                                                                                     \
    if (phase == ITER) {                                                                                  \
      if (df) return launch_iter<N_, float, df64>(L, arg_i);                                              \
      return qt32 ? launch_iter<N_, float, double>(L, arg_i) : launch_iter<N_, double, double>(L, arg_i); \
    }                                                                                                     \
    if (rows) return launch_rows<N_>(L, phase, arg_d, qt32);                                              \
    return df ? launch_aux<N_, df64>(L, phase, arg_i, qt32) : launch_aux<N_, double>(L, phase, arg_i, qt32);
    PGV_CASE(4)
    PGV_CASE(6)
    PGV_CASE(14)
#undef PGV_CASE
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace pgv

namespace {
thread_local std::string g_thread_error;
}  // namespace

void pgv::set_thread_error(const char* msg) { g_thread_error = msg ? msg : ""; }

using namespace pgv;

namespace {

pgvimp_status fail(std::string* where, pgvimp_status st, const std::string& msg) {
  g_thread_error = msg;
  if (where) *where = msg;
  return st;
}

constexpr int PH_PRIOR = 100, PH_INIT = 101, PH_ITER = 102, PH_SLR = 103, PH_RELIN = 104, PH_SLR_FIN = 105,
              PH_FINALIZE = 106, PH_WORKING = 107;

// ------------------------------------------------------------ GH rule tables
// Golub-Welsch: the nodes of the p-point rule for the N(0,1) weight are the
// eigenvalues of the Jacobi matrix of the probabilists' Hermite recurrence
// (zero diagonal, off-diagonal sqrt(k)); the weights are the squared first
// components of the normalised eigenvectors.  Cyclic Jacobi rotations.
void gh_golub_welsch(int p, double* x, double* w) {
  std::vector<double> J(p * p, 0.0), V(p * p, 0.0);
  for (int k = 0; k + 1 < p; ++k) J[k * p + k + 1] = J[(k + 1) * p + k] = std::sqrt((double)(k + 1));
  for (int i = 0; i < p; ++i) V[i * p + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) off += J[i * p + j] * J[i * p + j];
    if (off < 1e-40) break;
    for (int i = 0; i < p; ++i)
      for (int j = i + 1; j < p; ++j) {
        double aij = J[i * p + j];
        if (std::fabs(aij) < 1e-300) continue;
        double theta = (J[j * p + j] - J[i * p + i]) / (2.0 * aij);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < p; ++k) {
          double akp = J[k * p + i], akq = J[k * p + j];
          J[k * p + i] = c * akp - s * akq;
          J[k * p + j] = s * akp + c * akq;
        }
        for (int k = 0; k < p; ++k) {
          double apk = J[i * p + k], aqk = J[j * p + k];
          J[i * p + k] = c * apk - s * aqk;
          J[j * p + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < p; ++k) {
          double vkp = V[k * p + i], vkq = V[k * p + j];
          V[k * p + i] = c * vkp - s * vkq;
          V[k * p + j] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<std::pair<double, double>> nw(p);
  for (int i = 0; i < p; ++i) nw[i] = {J[i * p + i], V[0 * p + i] * V[0 * p + i]};
  std::sort(nw.begin(), nw.end());
  for (int i = 0; i < p; ++i) {
    x[i] = nw[i].first;
    w[i] = nw[i].second;
  }
  // exact symmetry of the rule
  for (int i = 0; i < p / 2; ++i) {
    double xs = 0.5 * (x[p - 1 - i] - x[i]), ws = 0.5 * (w[i] + w[p - 1 - i]);
    x[i] = -xs;
    x[p - 1 - i] = xs;
    w[i] = w[p - 1 - i] = ws;
  }
  if (p % 2) x[p / 2] = 0.0;
  double sum = 0.0;
  for (int i = 0; i < p; ++i) sum += w[i];
  for (int i = 0; i < p; ++i) w[i] /= sum;
}

std::mutex g_init_mu;
bool g_tables_ready = false;
double g_gh_x[(kMaxGH + 1) * kMaxGH], g_gh_w[(kMaxGH + 1) * kMaxGH];

// The rule tables travel with each batch's inputs (no device-global state).
void ensure_tables() {
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_tables_ready) return;
  std::memset(g_gh_x, 0, sizeof(g_gh_x));
  std::memset(g_gh_w, 0, sizeof(g_gh_w));
  for (int p = 1; p <= kMaxGH; ++p) gh_golub_welsch(p, g_gh_x + p * kMaxGH, g_gh_w + p * kMaxGH);
  g_tables_ready = true;
}

// ------------------------------------------------------------ sparse grids

// Smolyak sparse grid of level k over d dimensions (Lemma 1), built from the
// 1-D Gauss-Hermite rules with i = 1..k points by the combination formula
//   sum over multi-indices i >= 1 with d + max(0, k - d) <= |i| <= d + k - 1
//   of (-1)^(d + k - 1 - |i|) C(d - 1, d + k - 1 - |i|) U^{i_1} x ... x U^{i_d};
// exact for total degree 2k - 1.  Coinciding nodes (to 1e-12) are merged.
// `add` receives each (node, weight) of the combination.
struct GridKey {
  std::vector<long long> q;
  bool operator<(const GridKey& o) const { return q < o.q; }
};

void smolyak_terms(int d, int k, const std::function<void(const double*, double)>& add) {
  std::vector<int> idx(d, 1), dig(d, 0);
  std::vector<double> pt(d);
  const int top = d + k - 1, low = d + std::max(0, k - d);
  std::function<void(int, int)> rec = [&](int j, int sum) {
    if (j == d) {
      if (sum < low) return;
      const int m = top - sum;
      double c = (m % 2) ? -1.0 : 1.0;
      for (int t = 1; t <= m; ++t) c = c * (d - 1 - m + t) / t;   // C(d-1, m)
      std::fill(dig.begin(), dig.end(), 0);
      for (;;) {
        double w = c;
        for (int a = 0; a < d; ++a) {
          pt[a] = g_gh_x[idx[a] * kMaxGH + dig[a]];
          w *= g_gh_w[idx[a] * kMaxGH + dig[a]];
        }
        add(pt.data(), w);
        int a = d - 1;
        while (a >= 0 && ++dig[a] == idx[a]) dig[a--] = 0;
        if (a < 0) break;
      }
      return;
    }
    for (int i = 1; i <= k && sum + i + (d - 1 - j) <= top; ++i) {
      idx[j] = i;
      rec(j + 1, sum + i);
    }
  };
  rec(0, 0);
}

// Number of multi-indices and of (unmerged) nodes of the level-k grid.
void smolyak_size(int d, int k, double* terms, double* nodes) {
  *terms = 0.0;
  *nodes = 0.0;
  std::function<void(int, int, double)> rec = [&](int j, int sum, double prod) {
    if (*terms > 1e7) return;
    if (j == d) {
      if (sum >= d + std::max(0, k - d)) {
        *terms += 1.0;
        *nodes += prod;
      }
      return;
    }
    for (int i = 1; i <= k && sum + i + (d - 1 - j) <= d + k - 1; ++i) rec(j + 1, sum + i, prod * i);
  };
  rec(0, 0, 1.0);
}

// Merged table with `cols` weight columns: column c holds the level (k - c) grid.
std::vector<double> sparse_table(int d, int k, int cols) {
  ensure_tables();
  std::map<GridKey, std::vector<double>> pts;
  for (int c = 0; c < cols; ++c) {
    if (k - c < 1) continue;
    smolyak_terms(d, k - c, [&](const double* x, double w) {
      GridKey key;
      key.q.resize(d);
      for (int a = 0; a < d; ++a) key.q[a] = std::llround(x[a] * 1e12);
      auto it = pts.find(key);
      if (it == pts.end()) {
        std::vector<double> row(d + cols, 0.0);
        for (int a = 0; a < d; ++a) row[a] = x[a];
        it = pts.emplace(key, row).first;
      }
      it->second[d + c] += w;
    });
  }
  std::vector<double> out;
  out.reserve(pts.size() * (d + cols));
  for (auto& kv : pts) out.insert(out.end(), kv.second.begin(), kv.second.end());
  return out;
}

// ------------------------------------------------------------ validation

bool finite_all(const double* p, size_t k) {
  for (size_t i = 0; i < k; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}
bool spd(const double* A, int n) {
  std::vector<double> L(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (std::fabs(A[i * n + j] - A[j * n + i]) > 1e-9 * (std::fabs(A[i * n + j]) + std::fabs(A[j * n + i]) + 1e-300))
        return false;
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return false;
    L[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  return true;
}

bool supported_n(int n) { return n == 4 || n == 6 || n == 14; }

int cost_dims(const pgvimp_problem& p) {
  switch (p.cost_kind) {
    case PGVIMP_COST_POINT2D: return 2;
    case PGVIMP_COST_POINT3D: return 3;
    case PGVIMP_COST_ARM: return p.arm_dof;
    default: return 0;
  }
}

// `scan_grid` = false skips the per-cell finiteness scan of the SDF (for
// requests a server already validated at submit).
pgvimp_status validate(const pgvimp_problem& p, const pgvimp_options& o, int idx, std::string* err,
                       bool scan_grid = true) {
  auto E = [&](pgvimp_status st, const std::string& m) { return fail(err, st, "problem " + std::to_string(idx) + ": " + m); };
  if (!supported_n(p.n)) return E(PGVIMP_EINVAL, "state dimension n must be one of 4, 6, 14");
  if (p.m < 1 || p.m > kMaxN) return E(PGVIMP_EINVAL, "noise dimension m out of range");
  if (p.N < 1 || p.N > (1 << 22)) return E(PGVIMP_EINVAL, "N out of range");
  if (!(p.T > 0.0) || !std::isfinite(p.T)) return E(PGVIMP_EINVAL, "T must be positive and finite");
  if (!p.B || !p.Qc || !p.mu0 || !p.K0 || !p.muN || !p.KN) return E(PGVIMP_EINVAL, "missing B, Qc, mu0, K0, muN or KN");
  const int n = p.n, m = p.m;
  if (p.dyn_kind == PGVIMP_DYN_LINEAR) {
    if (!p.A) return E(PGVIMP_EINVAL, "missing A");
    if (!finite_all(p.A, (size_t)(p.A_per_step ? p.N : 1) * n * n)) return E(PGVIMP_ENOTFINITE, "A not finite");
  } else if (p.dyn_kind == PGVIMP_DYN_PLANAR_QUAD) {
    if (n != 6) return E(PGVIMP_EINVAL, "planar quadrotor needs n = 6");
    if (o.slr_iters < 1) return E(PGVIMP_EINVAL, "SLR model needs slr_iters >= 1");
    if (!finite_all(p.dyn_params, 4)) return E(PGVIMP_ENOTFINITE, "dyn_params not finite");
  } else {
    return E(PGVIMP_EINVAL, "unknown dyn_kind");
  }
  if (p.a && !finite_all(p.a, (size_t)(p.a_per_step ? p.N : 1) * n)) return E(PGVIMP_ENOTFINITE, "a not finite");
  if (!finite_all(p.B, (size_t)n * m) || !finite_all(p.Qc, (size_t)m * m) || !finite_all(p.mu0, n) ||
      !finite_all(p.muN, n) || !finite_all(p.K0, (size_t)n * n) || !finite_all(p.KN, (size_t)n * n))
    return E(PGVIMP_ENOTFINITE, "an input matrix is not finite");
  if (!spd(p.Qc, m)) return E(PGVIMP_ENOTPD, "Qc is not symmetric positive definite");
  if (!spd(p.K0, n)) return E(PGVIMP_ENOTPD, "K0 is not symmetric positive definite");
  if (!spd(p.KN, n)) return E(PGVIMP_ENOTPD, "KN is not symmetric positive definite");
  const int dc = cost_dims(p);
  if (p.cost_kind < 0 || p.cost_kind > PGVIMP_COST_ARM) return E(PGVIMP_EINVAL, "unknown cost_kind");
  if (dc > n / 2 && p.cost_kind != PGVIMP_COST_NONE && p.dyn_kind == PGVIMP_DYN_LINEAR && p.cost_kind != PGVIMP_COST_POINT2D)
    return E(PGVIMP_EINVAL, "cost dimensions exceed the configuration dimension");
  if (dc > n) return E(PGVIMP_EINVAL, "cost dimensions exceed n");
  if (p.cost_kind != PGVIMP_COST_NONE) {
    if (!(p.sigma_obs > 0.0) || !std::isfinite(p.sigma_obs) || !std::isfinite(p.eps))
      return E(PGVIMP_EINVAL, "sigma_obs must be positive, eps finite");
    if (!p.sdf || p.sdf_nx < 2 || p.sdf_ny < 2) return E(PGVIMP_EINVAL, "SDF grid missing or smaller than 2x2");
    const bool three = (p.cost_kind != PGVIMP_COST_POINT2D);
    if (three && p.sdf_nz < 2) return E(PGVIMP_EINVAL, "3-D cost needs sdf_nz >= 2");
    if (!(p.sdf_cell > 0.0) || !finite_all(p.sdf_origin, 3)) return E(PGVIMP_EINVAL, "bad SDF geometry");
    size_t cells = (size_t)p.sdf_nx * p.sdf_ny * (three ? p.sdf_nz : 1);
    for (size_t i = 0; scan_grid && i < cells; ++i)
      if (!std::isfinite(p.sdf[i])) return E(PGVIMP_ENOTFINITE, "SDF not finite");
  }
  if (p.cost_kind == PGVIMP_COST_ARM) {
    if (p.arm_dof < 1 || p.arm_dof > kMaxDof || p.arm_dof != n / 2) return E(PGVIMP_EINVAL, "arm_dof must equal n/2 and be <= 8");
    if (!p.arm_dh || !p.sphere_link || !p.sphere_off || !p.sphere_r) return E(PGVIMP_EINVAL, "missing arm model");
    if (p.n_spheres < 1 || p.n_spheres > kMaxSpheres) return E(PGVIMP_EINVAL, "n_spheres out of range");
    for (int k = 0; k < p.n_spheres; ++k)
      if (p.sphere_link[k] < 0 || p.sphere_link[k] >= p.arm_dof) return E(PGVIMP_EINVAL, "sphere_link out of range");
    if (!finite_all(p.arm_dh, 4 * p.arm_dof) || !finite_all(p.sphere_off, 3 * p.n_spheres) ||
        !finite_all(p.sphere_r, p.n_spheres))
      return E(PGVIMP_ENOTFINITE, "arm model not finite");
  }
  if (o.rule != PGVIMP_RULE_GH && o.rule != PGVIMP_RULE_DEG3 && o.rule != PGVIMP_RULE_SMOLYAK)
    return E(PGVIMP_EINVAL, "unknown rule");
  if (o.rule == PGVIMP_RULE_SMOLYAK) {
    if (o.gh_p < 2 || o.gh_p > kMaxGH) return E(PGVIMP_EINVAL, "Smolyak level (gh_p) must be in 2..10");
    double terms, nodes;
    smolyak_size(std::max(dc, p.dyn_kind != PGVIMP_DYN_LINEAR ? n : 0), o.gh_p, &terms, &nodes);
    if (terms > 1e5 || nodes > 2e5) return E(PGVIMP_EINVAL, "sparse grid too large");
  }
  if (o.rule == PGVIMP_RULE_GH) {
    if (o.gh_p < 2 || o.gh_p > kMaxGH) return E(PGVIMP_EINVAL, "gh_p must be in 2..10");
    double pts = std::pow((double)o.gh_p, (double)std::max(dc, p.dyn_kind != PGVIMP_DYN_LINEAR ? n : 0));
    if (pts > 2.0e6) return E(PGVIMP_EINVAL, "quadrature rule too large");
  }
  if (!(o.beta_max > 0.0) || !std::isfinite(o.beta_max)) return E(PGVIMP_EINVAL, "beta_max must be positive");
  if (!(o.kl_eps > 0.0)) return E(PGVIMP_EINVAL, "kl_eps must be positive (may be +inf)");
  if (o.max_bisect < 0 || o.max_bisect > 60) return E(PGVIMP_EINVAL, "max_bisect out of range");
  if (o.iters < 0 || o.iters > (1 << 20)) return E(PGVIMP_EINVAL, "iters out of range");
  if (o.init_kind == 1 && !(o.init_scale > 0.0)) return E(PGVIMP_EINVAL, "init_scale must be positive");
  if ((o.plan_threads > 1 && o.plan_threads != kLaneThreads &&
       (o.plan_threads < 32 || o.plan_threads > kCrMaxThreads || (o.plan_threads & 31))) || o.plan_threads < 0)
    return E(PGVIMP_EINVAL, "plan_threads must be 0, 1, 16, or a multiple of 32 in 32..256");
  if (o.plan_threads == kLaneThreads && p.n != 4)
    return E(PGVIMP_EINVAL, "the lane form (plan_threads = 16) is built for state dimension 4");
  if (!(o.temperature_high >= 0.0) || !std::isfinite(o.temperature_high) || o.switch_iter < 0)
    return E(PGVIMP_EINVAL, "temperature_high must be finite and >= 0, switch_iter >= 0");
  if (o.update != PGVIMP_UPDATE_PROX && o.update != PGVIMP_UPDATE_NGD) return E(PGVIMP_EINVAL, "unknown update");
  if (o.update == PGVIMP_UPDATE_NGD && o.beta_max > 1.0)
    return E(PGVIMP_EINVAL, "the natural-gradient step needs beta_max <= 1");
  return PGVIMP_OK;
}

// ------------------------------------------------------------ layout

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct PlanLayout {
  // offsets in bytes inside their sections
  size_t A, a, B, Qc, mu0, K0, muN, KN, dh, soff, srad, sdf;      // INPUT
  size_t mu0_, Sd0, So0, Ld, Lo;                                  // OUTPUT (per plan)
  size_t Kd, Ko, b, mubar, mu1, Sd1, So1, mu2, Sd2, So2, g, G, Altv, altv, xbar, scr;  // WORK
  size_t A_cnt, a_cnt, sdf_cnt;
  bool sdf_owner;   // false: the grid is shared with an earlier plan of the batch
  size_t sg, sgs;   // Smolyak tables (INPUT offsets), shared by plans with the same rule
  int sg_rows, sgs_rows;
  int log_cap, slr_cap;
};

struct BatchImpl {
  int count = 0, n = 0, precision = 0, dyn = 0;
  int tpb = 0;   // threads per plan in the block form (0: one thread per plan, or the lane form)
  bool lane = false;   // lane form of the fused iterations (n = 4: plan_threads 16, or 0 with double-float)
  int iters_opt = 0, slr_opt = 0;
  std::vector<pgvimp_problem> probs;
  std::vector<pgvimp_options> opts;
  std::vector<PlanLayout> lay;
  std::vector<PlanDesc> desc;
  // sparse-grid tables of the batch by (dimension, level, weight columns):
  // INPUT offset and contents
  std::map<std::tuple<int, int, int>, std::pair<size_t, std::vector<double>>> grids;
  size_t in_bytes = 0, res_bytes = 0, extra_bytes = 0, work_bytes = 0;
  size_t off_desc = 0, off_gh = 0, off_scal = 0, off_log = 0, off_slrn = 0;
  char* arena = nullptr;
  bool owns_arena = false;
  char* h_in = nullptr;   // pinned INPUT staging
  char* h_out = nullptr;  // pinned OUTPUT staging (result + extra)
  bool owns_host = true;  // false: the staging belongs to the caller (a server's pinned pool)
  bool started = false;
  int j_host = 0, kin_host = 0;
  std::string err;
  ~BatchImpl() {
    if (owns_arena && arena) cudaFree(arena);
    if (owns_host && h_in) cudaFreeHost(h_in);
    if (owns_host && h_out) cudaFreeHost(h_out);
  }
  char* d_in() const { return arena; }
  char* d_res() const { return arena + in_bytes; }
  char* d_extra() const { return arena + in_bytes + res_bytes; }
  char* d_work() const { return arena + in_bytes + res_bytes + extra_bytes; }
  size_t total() const { return in_bytes + res_bytes + extra_bytes + work_bytes; }
};

// Computes every offset; returns the section sizes.
void plan_layout(BatchImpl& B) {
  const int cnt = B.count;
  size_t in = align256(sizeof(PlanDesc) * cnt);
  B.off_desc = 0;
  B.off_gh = in;
  in = align256(in + 2 * sizeof(double) * (kMaxGH + 1) * kMaxGH);
  size_t res = 0;
  B.off_scal = res;
  res = align256(res + sizeof(double) * kScal * cnt);
  int log_cap = 0, slr_cap = 1;
  for (int i = 0; i < cnt; ++i) {
    const pgvimp_options& o = B.opts[i];
    int lc = o.iters * (B.dyn != PGVIMP_DYN_LINEAR ? std::max(o.slr_iters, 1) : 1);
    log_cap = std::max(log_cap, std::max(lc, 1));
    slr_cap = std::max(slr_cap, o.slr_iters);
  }
  B.off_log = res;
  res = align256(res + sizeof(pgvimp_step_info) * (size_t)log_cap * cnt);
  B.off_slrn = res;
  res = align256(res + sizeof(double) * (size_t)slr_cap * cnt);
  size_t extra = 0, work = 0;
  B.lay.resize(cnt);
  // Plans that pass the same host grid (same pointer and size) share one
  // device copy: maps are read-only and a batch often reuses a few of them.
  std::map<std::pair<const float*, size_t>, size_t> sdf_seen;
  for (int i = 0; i < cnt; ++i) {
    const pgvimp_problem& p = B.probs[i];
    PlanLayout& L = B.lay[i];
    const size_t n = p.n, m = p.m, N = p.N, nn = n * n;
    auto take = [](size_t& cur, size_t bytes) {
      size_t o = cur;
      cur = align256(cur + bytes);
      return o;
    };
    L.log_cap = log_cap;
    L.slr_cap = slr_cap;
    L.A_cnt = (p.dyn_kind == PGVIMP_DYN_LINEAR) ? (p.A_per_step ? N : 1) * nn : 0;
    L.a_cnt = p.a ? (p.a_per_step ? N : 1) * n : 0;
    const bool three = (p.cost_kind == PGVIMP_COST_POINT3D || p.cost_kind == PGVIMP_COST_ARM);
    L.sdf_cnt = (p.cost_kind == PGVIMP_COST_NONE) ? 0 : (size_t)p.sdf_nx * p.sdf_ny * (three ? p.sdf_nz : 1);
    L.A = take(in, 8 * std::max<size_t>(L.A_cnt, 1));
    L.a = take(in, 8 * std::max<size_t>(L.a_cnt, 1));
    L.B = take(in, 8 * n * m);
    L.Qc = take(in, 8 * m * m);
    L.mu0 = take(in, 8 * n);
    L.K0 = take(in, 8 * nn);
    L.muN = take(in, 8 * n);
    L.KN = take(in, 8 * nn);
    const size_t dof = (p.cost_kind == PGVIMP_COST_ARM) ? p.arm_dof : 0, S = dof ? p.n_spheres : 0;
    L.dh = take(in, 8 * std::max<size_t>(4 * dof, 1));
    L.soff = take(in, 8 * std::max<size_t>(3 * S, 1));
    L.srad = take(in, 8 * std::max<size_t>(S, 1));
    L.sg = L.sgs = 0;
    L.sg_rows = L.sgs_rows = 0;
    if (B.opts[i].rule == PGVIMP_RULE_SMOLYAK) {
      auto table = [&](int d, int k, int cols, size_t* off, int* rows) {
        auto key = std::make_tuple(d, k, cols);
        auto it = B.grids.find(key);
        if (it == B.grids.end()) {
          std::vector<double> t = sparse_table(d, k, cols);
          size_t o = take(in, 8 * std::max<size_t>(t.size(), 2));
          it = B.grids.emplace(key, std::make_pair(o, std::move(t))).first;
        }
        *off = it->second.first;
        *rows = (int)(it->second.second.size() / (d + cols));
      };
      const int dc = cost_dims(p);
      if (p.cost_kind != PGVIMP_COST_NONE && dc > 0) table(dc, B.opts[i].gh_p, 2, &L.sg, &L.sg_rows);
      if (p.dyn_kind != PGVIMP_DYN_LINEAR) table((int)n, B.opts[i].gh_p, 1, &L.sgs, &L.sgs_rows);
    }
    L.sdf_owner = true;
    if (L.sdf_cnt) {
      auto key = std::make_pair(p.sdf, L.sdf_cnt);
      auto it = sdf_seen.find(key);
      if (it != sdf_seen.end()) {
        L.sdf = it->second;
        L.sdf_owner = false;
      } else {
        L.sdf = take(in, 4 * L.sdf_cnt);
        sdf_seen.emplace(key, L.sdf);
      }
    } else {
      L.sdf = take(in, 4);
    }
    L.mu0_ = take(res, 8 * (N + 1) * n);
    L.Sd0 = take(res, 8 * (N + 1) * nn);
    L.So0 = take(extra, 8 * N * nn);
    L.Ld = take(extra, 8 * (N + 1) * nn);
    L.Lo = take(extra, 8 * N * nn);
    L.Kd = take(work, 8 * (N + 1) * nn);
    L.Ko = take(work, 8 * N * nn);
    L.b = take(work, 8 * (N + 1) * n);
    L.mubar = take(work, 8 * (N + 1) * n);
    L.mu1 = take(work, 8 * (N + 1) * n);
    L.Sd1 = take(work, 8 * (N + 1) * nn);
    L.So1 = take(work, 8 * N * nn);
    L.mu2 = take(work, 8 * (N + 1) * n);
    L.Sd2 = take(work, 8 * (N + 1) * nn);
    L.So2 = take(work, 8 * N * nn);
    L.g = take(work, 8 * (N + 1) * n);
    L.G = take(work, 8 * (N + 1) * nn);
    const bool slr = p.dyn_kind != PGVIMP_DYN_LINEAR;
    L.Altv = take(work, 8 * (slr ? N * nn : 1));
    L.altv = take(work, 8 * (slr ? N * n : 1));
    L.xbar = take(work, 8 * (slr ? (N + 1) * n : 1));
    // per-state scratch: the sequential sweeps need 3n^2 + n, the cyclic
    // reduction of the block form 2 npe + 6 n^2 + 2 n (npe: packed, even),
    // its warp-cooperative form 8 n^2 + 2 n
    const size_t np = n * (n + 1) / 2, npe = np + (np & 1);
    const size_t scr_state =
        B.tpb ? std::max(std::max(3 * nn + n, 2 * npe + 6 * nn + 2 * n), 8 * nn + 2 * n) : 3 * nn + n;
    L.scr = take(work, 8 * (N + 1) * scr_state);
  }
  B.in_bytes = align256(in);
  B.res_bytes = align256(res);
  B.extra_bytes = align256(extra);
  B.work_bytes = align256(work);
}

void build_descs(BatchImpl& B) {
  B.desc.resize(B.count);
  char* din = B.d_in();
  char* dres = B.d_res();
  char* dext = B.d_extra();
  char* dwork = B.d_work();
  for (int i = 0; i < B.count; ++i) {
    const pgvimp_problem& p = B.probs[i];
    const pgvimp_options& o = B.opts[i];
    const PlanLayout& L = B.lay[i];
    PlanDesc d;
    std::memset(&d, 0, sizeof(d));
    d.n = p.n; d.m = p.m; d.N = p.N; d.nq = p.n / 2; d.dc = cost_dims(p);
    d.T = p.T; d.dt = p.T / p.N;
    d.rule = o.rule; d.gh_p = o.gh_p; d.max_bisect = o.max_bisect; d.iters = o.iters;
    d.slr_iters = o.slr_iters; d.init_kind = o.init_kind; d.update = o.update;
    d.beta_max = o.beta_max; d.kl_eps = o.kl_eps; d.init_scale = o.init_scale;
    d.cost_kind = p.cost_kind; d.psi_form = p.psi_form; d.factor_set = p.factor_set;
    d.eps = p.eps; d.sigma_obs = p.sigma_obs; d.inv_temp = (p.temperature > 0.0) ? 1.0 / p.temperature : 1.0;
    d.inv_temp_high = (o.temperature_high > 0.0 && o.switch_iter > 0) ? 1.0 / o.temperature_high : 0.0;
    d.switch_iter = o.switch_iter;
    d.nx = p.sdf_nx; d.ny = p.sdf_ny; d.nz = std::max(p.sdf_nz, 1);
    for (int k = 0; k < 3; ++k) d.sdf_origin[k] = p.sdf_origin[k];
    d.cell = p.sdf_cell; d.inv_cell = p.sdf_cell > 0 ? 1.0 / p.sdf_cell : 0.0;
    d.sdf = reinterpret_cast<const float*>(din + L.sdf);
    d.arm_dof = (p.cost_kind == PGVIMP_COST_ARM) ? p.arm_dof : 0;
    d.n_spheres = d.arm_dof ? p.n_spheres : 0;
    d.dh = reinterpret_cast<const double*>(din + L.dh);
    d.sphere_off = reinterpret_cast<const double*>(din + L.soff);
    d.sphere_r = reinterpret_cast<const double*>(din + L.srad);
    if (d.arm_dof) {
      int c = 0;
      for (int j = 0; j <= d.arm_dof; ++j) {
        d.sphere_begin[j] = c;
        if (j < d.arm_dof)
          for (int k = 0; k < p.n_spheres; ++k) c += (p.sphere_link[k] == j);
      }
    }
    d.sg = reinterpret_cast<const double*>(din + L.sg);
    d.sgs = reinterpret_cast<const double*>(din + L.sgs);
    d.sg_rows = L.sg_rows;
    d.sgs_rows = L.sgs_rows;
    d.gh_x = reinterpret_cast<const double*>(din + B.off_gh);
    d.gh_w = d.gh_x + (kMaxGH + 1) * kMaxGH;
    d.dyn_kind = p.dyn_kind;
    for (int k = 0; k < 4; ++k) d.dyn_params[k] = p.dyn_params[k];
    d.A = reinterpret_cast<const double*>(din + L.A);
    d.a = L.a_cnt ? reinterpret_cast<const double*>(din + L.a) : nullptr;
    d.A_per_step = p.A_per_step; d.a_per_step = p.a_per_step;
    d.B = reinterpret_cast<const double*>(din + L.B);
    d.Qc = reinterpret_cast<const double*>(din + L.Qc);
    d.mu0 = reinterpret_cast<const double*>(din + L.mu0);
    d.K0 = reinterpret_cast<const double*>(din + L.K0);
    d.muN = reinterpret_cast<const double*>(din + L.muN);
    d.KN = reinterpret_cast<const double*>(din + L.KN);
    auto W = [&](size_t off) { return reinterpret_cast<double*>(dwork + off); };
    d.Kd = W(L.Kd); d.Ko = W(L.Ko); d.b = W(L.b); d.mubar = W(L.mubar);
    d.Ld = reinterpret_cast<double*>(dext + L.Ld);
    d.Lo = reinterpret_cast<double*>(dext + L.Lo);
    d.mu[0] = reinterpret_cast<double*>(dres + L.mu0_);
    d.Sd[0] = reinterpret_cast<double*>(dres + L.Sd0);
    d.So[0] = reinterpret_cast<double*>(dext + L.So0);
    d.mu[1] = W(L.mu1); d.Sd[1] = W(L.Sd1); d.So[1] = W(L.So1);
    d.mu[2] = W(L.mu2); d.Sd[2] = W(L.Sd2); d.So[2] = W(L.So2);
    d.g = W(L.g); d.G = W(L.G);
    d.Altv = W(L.Altv); d.altv = W(L.altv); d.xbar = W(L.xbar);
    d.scr = W(L.scr);
    d.scal = reinterpret_cast<double*>(dres + B.off_scal) + (size_t)kScal * i;
    d.slr_norms = reinterpret_cast<double*>(dres + B.off_slrn) + (size_t)L.slr_cap * i;
    d.log = reinterpret_cast<pgvimp_step_info*>(dres + B.off_log) + (size_t)L.log_cap * i;
    d.log_cap = L.log_cap;
    B.desc[i] = d;
  }
}

void stage_inputs(BatchImpl& B) {
  char* h = B.h_in;
  std::memcpy(h + B.off_desc, B.desc.data(), sizeof(PlanDesc) * B.count);
  std::memcpy(h + B.off_gh, g_gh_x, sizeof(g_gh_x));
  std::memcpy(h + B.off_gh + sizeof(g_gh_x), g_gh_w, sizeof(g_gh_w));
  for (auto& kv : B.grids)
    if (!kv.second.second.empty())
      std::memcpy(h + kv.second.first, kv.second.second.data(), 8 * kv.second.second.size());
  for (int i = 0; i < B.count; ++i) {
    const pgvimp_problem& p = B.probs[i];
    const PlanLayout& L = B.lay[i];
    const size_t n = p.n, m = p.m, nn = n * n;
    if (L.A_cnt) std::memcpy(h + L.A, p.A, 8 * L.A_cnt);
    if (L.a_cnt) std::memcpy(h + L.a, p.a, 8 * L.a_cnt);
    std::memcpy(h + L.B, p.B, 8 * n * m);
    std::memcpy(h + L.Qc, p.Qc, 8 * m * m);
    std::memcpy(h + L.mu0, p.mu0, 8 * n);
    std::memcpy(h + L.K0, p.K0, 8 * nn);
    std::memcpy(h + L.muN, p.muN, 8 * n);
    std::memcpy(h + L.KN, p.KN, 8 * nn);
    if (p.cost_kind == PGVIMP_COST_ARM) {
      std::memcpy(h + L.dh, p.arm_dh, 8 * 4 * p.arm_dof);
      // spheres grouped by link (the cost is a sum over spheres)
      int c = 0;
      double* off = reinterpret_cast<double*>(h + L.soff);
      double* rad = reinterpret_cast<double*>(h + L.srad);
      for (int j = 0; j < p.arm_dof; ++j)
        for (int k = 0; k < p.n_spheres; ++k)
          if (p.sphere_link[k] == j) {
            off[3 * c] = p.sphere_off[3 * k];
            off[3 * c + 1] = p.sphere_off[3 * k + 1];
            off[3 * c + 2] = p.sphere_off[3 * k + 2];
            rad[c] = p.sphere_r[k];
            ++c;
          }
    }
    if (L.sdf_cnt && L.sdf_owner) std::memcpy(h + L.sdf, p.sdf, 4 * L.sdf_cnt);
  }
}

pgvimp_status cuda_fail(std::string* err, cudaError_t e, const char* what) {
  return fail(err, PGVIMP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

pgvimp_status launch(BatchImpl& B, int phase, int arg_i, double arg_d, cudaStream_t s) {
  Launch L{reinterpret_cast<const PlanDesc*>(B.d_in() + B.off_desc), B.count, s};
  cudaError_t e = launch_phase(B.n, L, phase, arg_i, arg_d, B.precision, B.tpb, B.lane);
  if (e != cudaSuccess) return cuda_fail(&B.err, e, "kernel launch");
  return PGVIMP_OK;
}

}  // namespace

struct pgvimp_batch : BatchImpl {};

struct pgvimp_ctx {
  pgvimp_batch* b = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

extern "C" {

pgvimp_status pgvimp_version(char* buf, size_t len) {
  if (!buf || !len) return PGVIMP_EINVAL;
  int dev = -1;
  cudaDeviceProp pr;
  std::string s = "pgvimp b300 (sm_103a)";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&pr, dev) == cudaSuccess)
    s += std::string(" on ") + pr.name;
  std::snprintf(buf, len, "%s", s.c_str());
  return PGVIMP_OK;
}

pgvimp_status pgvimp_abi_sizes(size_t* problem, size_t* options, size_t* step_info) {
  if (problem) *problem = sizeof(pgvimp_problem);
  if (options) *options = sizeof(pgvimp_options);
  if (step_info) *step_info = sizeof(pgvimp_step_info);
  return PGVIMP_OK;
}

const char* pgvimp_last_error(const void* ctx) {
  (void)ctx;
  return g_thread_error.c_str();
}

static pgvimp_status prepare(int count, const pgvimp_problem* problems, const pgvimp_options* options, int precision,
                             BatchImpl& B, bool scan_grids = true) {
  if (count < 1 || !problems || !options) return fail(&B.err, PGVIMP_EINVAL, "count must be >= 1 with problems and options");
  if (precision != PGVIMP_PREC_PLAIN_FP64 && precision != PGVIMP_PREC_MIXED && precision != PGVIMP_PREC_MIXED_DF)
    return fail(&B.err, PGVIMP_EINVAL, "unknown precision");
  std::set<const float*> scanned;   // a grid shared by several plans is scanned once
  for (int i = 0; i < count; ++i) {
    const bool scan = scan_grids && scanned.insert(problems[i].sdf).second;
    pgvimp_status st = validate(problems[i], options[i], i, &B.err, scan);
    if (st != PGVIMP_OK) return st;
    if (problems[i].n != problems[0].n) return fail(&B.err, PGVIMP_EINVAL, "a batch needs one state dimension");
    if (problems[i].dyn_kind != problems[0].dyn_kind) return fail(&B.err, PGVIMP_EINVAL, "a batch needs one dynamics kind");
    if (options[i].plan_threads != options[0].plan_threads)
      return fail(&B.err, PGVIMP_EINVAL, "a batch needs one plan_threads");
    if (problems[i].dyn_kind != PGVIMP_DYN_LINEAR &&
        (options[i].iters != options[0].iters || options[i].slr_iters != options[0].slr_iters))
      return fail(&B.err, PGVIMP_EINVAL, "an SLR batch needs one iters / slr_iters");
  }
  B.count = count;
  B.n = problems[0].n;
  B.dyn = problems[0].dyn_kind;
  B.precision = precision;
  B.tpb = options[0].plan_threads >= 32 ? options[0].plan_threads : 0;
  // the default throughput form: the lane form where it is faster (n = 4 with
  // double-float recursions, whose FP32 pipe absorbs the lane form's extra
  // work; with FP64 recursions one thread per plan keeps the FP64 pipe busier)
  B.lane = options[0].plan_threads == kLaneThreads ||
           (options[0].plan_threads == 0 && B.n == 4 && precision == PGVIMP_PREC_MIXED_DF);
  B.iters_opt = options[0].iters;
  B.slr_opt = options[0].slr_iters;
  B.probs.assign(problems, problems + count);
  B.opts.assign(options, options + count);
  plan_layout(B);
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_arena_bytes(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                                       int precision, size_t* bytes) {
  if (!bytes) return fail(nullptr, PGVIMP_EINVAL, "bytes is NULL");
  BatchImpl B;
  pgvimp_status st = prepare(count, problems, options, precision, B);
  if (st != PGVIMP_OK) return st;
  *bytes = B.total();
  return PGVIMP_OK;
}

static pgvimp_status create_batch(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                                  int precision, void* arena, size_t arena_bytes, void* h_in, void* h_out,
                                  pgvimp_batch** out, bool scan_grids = true) {
  if (!out) return fail(nullptr, PGVIMP_EINVAL, "out is NULL");
  *out = nullptr;
  pgvimp_batch* B = new (std::nothrow) pgvimp_batch();
  if (!B) return fail(nullptr, PGVIMP_ENOMEM, "host allocation failed");
  pgvimp_status st = prepare(count, problems, options, precision, *B, scan_grids);
  ensure_tables();
  if (st != PGVIMP_OK) {
    delete B;
    return st;
  }
  const size_t total = B->total();
  if (arena) {
    if (arena_bytes < total) {
      delete B;
      return fail(nullptr, PGVIMP_ENOMEM, "arena smaller than pgvimp_batch_arena_bytes");
    }
    if (reinterpret_cast<uintptr_t>(arena) & 255) {
      delete B;
      return fail(nullptr, PGVIMP_EINVAL, "arena must be 256-byte aligned");
    }
    B->arena = static_cast<char*>(arena);
  } else {
    cudaError_t e = cudaMalloc(&B->arena, total);
    if (e != cudaSuccess) {
      delete B;
      return fail(nullptr, PGVIMP_ENOMEM, std::string("device arena: ") + cudaGetErrorString(e));
    }
    B->owns_arena = true;
  }
  if (h_in && h_out) {
    B->h_in = static_cast<char*>(h_in);
    B->h_out = static_cast<char*>(h_out);
    B->owns_host = false;
  } else if (cudaMallocHost(&B->h_in, B->in_bytes) != cudaSuccess ||
             cudaMallocHost(&B->h_out, B->res_bytes + B->extra_bytes) != cudaSuccess) {
    delete B;
    return fail(nullptr, PGVIMP_ENOMEM, "pinned host staging allocation failed");
  }
  build_descs(*B);
  stage_inputs(*B);
  // problem pointers refer to caller memory: forget them
  for (auto& p : B->probs) {
    p.A = p.a = p.B = p.Qc = p.mu0 = p.K0 = p.muN = p.KN = nullptr;
    p.sdf = nullptr;
    p.arm_dh = p.sphere_off = p.sphere_r = nullptr;
    p.sphere_link = nullptr;
  }
  *out = B;
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_create(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                                  int precision, void* arena, size_t arena_bytes, pgvimp_batch** out) {
  return create_batch(count, problems, options, precision, arena, arena_bytes, nullptr, nullptr, out);
}

pgvimp_status pgvimp_batch_upload(pgvimp_batch* b, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaError_t e = cudaMemcpyAsync(b->d_in(), b->h_in, b->in_bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&b->err, e, "upload");
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_reset(pgvimp_batch* b, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaError_t e = cudaMemsetAsync(b->d_res() + b->off_scal, 0, sizeof(double) * kScal * b->count, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&b->err, e, "reset");
  b->started = false;
  b->j_host = 0;
  b->kin_host = 0;
  return PGVIMP_OK;
}

static pgvimp_status finalize(pgvimp_batch* b, cudaStream_t s);

pgvimp_status pgvimp_batch_run(pgvimp_batch* b, int iters, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  pgvimp_status st;
  if (b->started && b->precision == PGVIMP_PREC_MIXED_DF && (st = launch(*b, PH_WORKING, 0, 0.0, s))) return st;
  if (b->dyn == PGVIMP_DYN_LINEAR) {
    if (!b->started) {
      if ((st = launch(*b, PH_PRIOR, 0, 0.0, s))) return st;
      if ((st = launch(*b, PH_INIT, 0, 0.0, s))) return st;
      b->started = true;
    }
    int max_it = 0;
    for (auto& o : b->opts) max_it = std::max(max_it, o.iters);
    int todo = iters <= 0 ? max_it : iters;
    if (todo > 0 && (st = launch(*b, PH_ITER, todo, 0.0, s))) return st;
    return finalize(b, s);
  }
  // Alg. 2: relinearise at the start of each outer iteration
  const int J = b->slr_opt, K = b->iters_opt;
  long remaining = iters <= 0 ? (long)J * K : iters;
  while (remaining > 0 && b->j_host < J) {
    if (b->kin_host == 0) {
      if (b->j_host == 0) {
        if ((st = launch(*b, PH_SLR, 1, 0.0, s))) return st;
        if ((st = launch(*b, PH_PRIOR, 1, 0.0, s))) return st;
        if ((st = launch(*b, PH_INIT, 0, 0.0, s))) return st;
        b->started = true;
      } else {
        if ((st = launch(*b, PH_SLR, 0, 0.0, s))) return st;
        if ((st = launch(*b, PH_PRIOR, 1, 0.0, s))) return st;
        if ((st = launch(*b, PH_RELIN, 0, 0.0, s))) return st;
      }
    }
    int step = (int)std::min<long>(remaining, K - b->kin_host);
    if (step > 0 && (st = launch(*b, PH_ITER, step, 0.0, s))) return st;
    b->kin_host += step;
    remaining -= step;
    if (b->kin_host >= K) {
      b->kin_host = 0;
      b->j_host += 1;
      if (b->j_host == J && (st = launch(*b, PH_SLR_FIN, 0, 0.0, s))) return st;
    }
    if (K == 0) break;
  }
  return finalize(b, s);
}

pgvimp_status pgvimp_batch_phase(pgvimp_batch* b, int phase, double arg, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  pgvimp_status st;
  if (b->precision == PGVIMP_PREC_MIXED_DF && phase != PGVIMP_PHASE_PRIOR)
    return fail(&b->err, PGVIMP_EINVAL, "single-row phases run with FP64 or mixed recursions only");
  switch (phase) {
    case PGVIMP_PHASE_PRIOR:
      if (b->dyn != PGVIMP_DYN_LINEAR) {
        if ((st = launch(*b, PH_SLR, 1, 0.0, s))) return st;
        if ((st = launch(*b, PH_PRIOR, 1, 0.0, s))) return st;
      } else if ((st = launch(*b, PH_PRIOR, 0, 0.0, s))) {
        return st;
      }
      if ((st = launch(*b, PH_INIT, 0, 0.0, s))) return st;
      b->started = true;
      return PGVIMP_OK;
    case PGVIMP_PHASE_MARGINALS:
    case PGVIMP_PHASE_QUAD:
    case PGVIMP_PHASE_TRIAL:
      return launch(*b, phase, 0, arg, s);
    case PGVIMP_PHASE_SLR:
      if (b->dyn == PGVIMP_DYN_LINEAR) return fail(&b->err, PGVIMP_EINVAL, "SLR phase needs a nonlinear model");
      return launch(*b, PH_SLR, 2, 0.0, s);
    default:
      return fail(&b->err, PGVIMP_EINVAL, "unknown phase");
  }
}

pgvimp_status pgvimp_batch_download(pgvimp_batch* b, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaError_t e = cudaMemcpyAsync(b->h_out, b->d_res(), b->res_bytes + b->extra_bytes, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&b->err, e, "download");
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_download_results(pgvimp_batch* b, void* stream) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  cudaError_t e = cudaMemcpyAsync(b->h_out, b->d_res(), b->res_bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(&b->err, e, "download");
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_io_bytes(const pgvimp_batch* b, size_t* h2d, size_t* d2h, size_t* d2h_results) {
  if (!b) return fail(nullptr, PGVIMP_EINVAL, "batch is NULL");
  if (h2d) *h2d = b->in_bytes;
  if (d2h) *d2h = b->res_bytes + b->extra_bytes;
  if (d2h_results) *d2h_results = b->res_bytes;
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_result(const pgvimp_batch* b, int index, double* mu, double* Sd, double* So, double* Ld,
                                  double* Lo, pgvimp_step_info* logs, int max_logs, int* n_logs) {
  if (!b || index < 0 || index >= b->count) return fail(nullptr, PGVIMP_EINVAL, "bad batch or index");
  const pgvimp_problem& p = b->probs[index];
  const PlanLayout& L = b->lay[index];
  const size_t n = p.n, N = p.N, nn = n * n;
  const char* hr = b->h_out;
  const char* he = b->h_out + b->res_bytes;
  if (mu) std::memcpy(mu, hr + L.mu0_, 8 * (N + 1) * n);
  if (Sd) std::memcpy(Sd, hr + L.Sd0, 8 * (N + 1) * nn);
  if (So) std::memcpy(So, he + L.So0, 8 * N * nn);
  if (Ld) std::memcpy(Ld, he + L.Ld, 8 * (N + 1) * nn);
  if (Lo) std::memcpy(Lo, he + L.Lo, 8 * N * nn);
  const double* sc = reinterpret_cast<const double*>(hr + b->off_scal) + (size_t)kScal * index;
  int k = (int)sc[S_K];
  int nl = std::min(k, L.log_cap);
  if (n_logs) *n_logs = nl;
  if (logs && max_logs > 0) {
    const pgvimp_step_info* src = reinterpret_cast<const pgvimp_step_info*>(hr + b->off_log) + (size_t)L.log_cap * index;
    std::memcpy(logs, src, sizeof(pgvimp_step_info) * std::min(nl, max_logs));
  }
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_destroy(pgvimp_batch* b) {
  delete b;
  return PGVIMP_OK;
}

// Device location and element count of a plan buffer; `pairs` tells whether
// it currently holds double-float pairs (double-float storage) or FP64.
static pgvimp_status resolve(const pgvimp_batch* b, int index, int buffer, double** dptr, size_t* cnt,
                             bool* pairs) {
  if (!b || index < 0 || index >= b->count) return fail(nullptr, PGVIMP_EINVAL, "bad batch or index");
  const PlanDesc& d = b->desc[index];
  const size_t n = d.n, N = d.N, nn = n * n;
  double scal[kScal];
  cudaError_t e = cudaMemcpy(scal, d.scal, sizeof(scal), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(nullptr, PGVIMP_ECUDA, std::string("read scalars: ") + cudaGetErrorString(e));
  const bool result_fp64 = scal[S_FMT] == 1.0 &&
                           (buffer == PGVIMP_BUF_MU || buffer == PGVIMP_BUF_SD || buffer == PGVIMP_BUF_SO ||
                            buffer == PGVIMP_BUF_LD || buffer == PGVIMP_BUF_LO);
  *pairs = b->precision == PGVIMP_PREC_MIXED_DF && buffer != PGVIMP_BUF_SCAL && buffer != PGVIMP_BUF_ALTV &&
           buffer != PGVIMP_BUF_ALTVA && !result_fp64;
  const int cur = (int)scal[S_CUR] % 3, tr = (cur + 2) % 3;
  switch (buffer) {
    case PGVIMP_BUF_MU: *dptr = d.mu[cur]; *cnt = (N + 1) * n; break;
    case PGVIMP_BUF_LD: *dptr = d.Ld; *cnt = (N + 1) * nn; break;
    case PGVIMP_BUF_LO: *dptr = d.Lo; *cnt = N * nn; break;
    case PGVIMP_BUF_SD: *dptr = d.Sd[cur]; *cnt = (N + 1) * nn; break;
    case PGVIMP_BUF_SO: *dptr = d.So[cur]; *cnt = N * nn; break;
    case PGVIMP_BUF_KD: *dptr = d.Kd; *cnt = (N + 1) * nn; break;
    case PGVIMP_BUF_KO: *dptr = d.Ko; *cnt = N * nn; break;
    case PGVIMP_BUF_B: *dptr = d.b; *cnt = (N + 1) * n; break;
    case PGVIMP_BUF_G1: *dptr = d.g; *cnt = (N + 1) * n; break;
    case PGVIMP_BUF_G2: *dptr = d.G; *cnt = (N + 1) * nn; break;
    case PGVIMP_BUF_TMU: *dptr = d.mu[tr]; *cnt = (N + 1) * n; break;
    case PGVIMP_BUF_TSD: *dptr = d.Sd[tr]; *cnt = (N + 1) * nn; break;
    case PGVIMP_BUF_TSO: *dptr = d.So[tr]; *cnt = N * nn; break;
    case PGVIMP_BUF_ALTV:
      if (d.dyn_kind == PGVIMP_DYN_LINEAR) return fail(nullptr, PGVIMP_EINVAL, "no SLR buffers for a linear model");
      *dptr = d.Altv; *cnt = N * nn; break;
    case PGVIMP_BUF_ALTVA:
      if (d.dyn_kind == PGVIMP_DYN_LINEAR) return fail(nullptr, PGVIMP_EINVAL, "no SLR buffers for a linear model");
      *dptr = d.altv; *cnt = N * n; break;
    case PGVIMP_BUF_SCAL: *dptr = d.scal; *cnt = kScal; break;
    default: return fail(nullptr, PGVIMP_EINVAL, "unknown buffer");
  }
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_read(const pgvimp_batch* b, int index, int buffer, double* host, size_t count) {
  double* d;
  size_t c;
  bool pairs;
  pgvimp_status st = resolve(b, index, buffer, &d, &c, &pairs);
  if (st) return st;
  if (!host || count != c) return fail(nullptr, PGVIMP_EINVAL, "count does not match the buffer size");
  cudaError_t e = cudaMemcpy(host, d, 8 * c, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(nullptr, PGVIMP_ECUDA, std::string("read: ") + cudaGetErrorString(e));
  if (pairs)
    for (size_t k = 0; k < c; ++k) {
      float hl[2];
      std::memcpy(hl, host + k, sizeof(hl));
      host[k] = (double)hl[0] + (double)hl[1];
    }
  return PGVIMP_OK;
}

pgvimp_status pgvimp_batch_write(pgvimp_batch* b, int index, int buffer, const double* host, size_t count) {
  double* d;
  size_t c;
  bool pairs;
  pgvimp_status st = resolve(b, index, buffer, &d, &c, &pairs);
  if (st) return st;
  if (!host || count != c) return fail(nullptr, PGVIMP_EINVAL, "count does not match the buffer size");
  std::vector<double> tmp;
  const double* src = host;
  if (pairs) {
    tmp.resize(c);
    for (size_t k = 0; k < c; ++k) {
      float hl[2];
      hl[0] = (float)host[k];
      hl[1] = (float)(host[k] - (double)hl[0]);
      std::memcpy(&tmp[k], hl, sizeof(hl));
    }
    src = tmp.data();
  }
  cudaError_t e = cudaMemcpy(d, src, 8 * c, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(nullptr, PGVIMP_ECUDA, std::string("write: ") + cudaGetErrorString(e));
  return PGVIMP_OK;
}

// ------------------------------------------------------------ context

pgvimp_status pgvimp_create(const pgvimp_problem* problem, const pgvimp_options* options, int precision,
                            pgvimp_ctx** out) {
  if (!out || !problem || !options) return fail(nullptr, PGVIMP_EINVAL, "NULL argument");
  *out = nullptr;
  pgvimp_ctx* c = new (std::nothrow) pgvimp_ctx();
  if (!c) return fail(nullptr, PGVIMP_ENOMEM, "host allocation failed");
  pgvimp_status st = pgvimp_batch_create(1, problem, options, precision, nullptr, 0, &c->b);
  if (st != PGVIMP_OK) {
    delete c;
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    pgvimp_batch_destroy(c->b);
    delete c;
    return fail(nullptr, PGVIMP_ECUDA, "stream creation failed");
  }
  if ((st = pgvimp_batch_upload(c->b, c->stream)) || (st = pgvimp_batch_reset(c->b, c->stream))) {
    pgvimp_destroy(c);
    return st;
  }
  *out = c;
  return PGVIMP_OK;
}

pgvimp_status pgvimp_step(pgvimp_ctx* c, pgvimp_step_info* info) {
  if (!c) return fail(nullptr, PGVIMP_EINVAL, "ctx is NULL");
  pgvimp_status st = pgvimp_batch_run(c->b, 1, c->stream);
  if (st) return st;
  if (info) {
    if ((st = pgvimp_batch_download(c->b, c->stream))) return st;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(&c->err, PGVIMP_ECUDA, cudaGetErrorString(e));
    const PlanLayout& L = c->b->lay[0];
    const double* sc = reinterpret_cast<const double*>(c->b->h_out + c->b->off_scal);
    int k = (int)sc[S_K];
    if (k >= 1 && k <= L.log_cap)
      *info = reinterpret_cast<const pgvimp_step_info*>(c->b->h_out + c->b->off_log)[k - 1];
    else
      std::memset(info, 0, sizeof(*info));
  }
  return PGVIMP_OK;
}

pgvimp_status pgvimp_plan(pgvimp_ctx* c, int iters) {
  if (!c) return fail(nullptr, PGVIMP_EINVAL, "ctx is NULL");
  pgvimp_status st = pgvimp_batch_run(c->b, iters, c->stream);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(&c->err, PGVIMP_ECUDA, cudaGetErrorString(e));
  return PGVIMP_OK;
}

pgvimp_status pgvimp_get(pgvimp_ctx* c, double* mu, double* Sigma, double* Lam_diag, double* Lam_off) {
  if (!c) return fail(nullptr, PGVIMP_EINVAL, "ctx is NULL");
  pgvimp_status st = pgvimp_batch_download(c->b, c->stream);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fail(&c->err, PGVIMP_ECUDA, cudaGetErrorString(e));
  return pgvimp_batch_result(c->b, 0, mu, Sigma, nullptr, Lam_diag, Lam_off, nullptr, 0, nullptr);
}

pgvimp_status pgvimp_destroy(pgvimp_ctx* c) {
  if (!c) return PGVIMP_OK;
  if (c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  pgvimp_batch_destroy(c->b);
  delete c;
  return PGVIMP_OK;
}

}  // extern "C"

// ---- internal entry points for the server (pgvimp_internal.h)
pgvimp_status pgv::batch_sizes(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                               int precision, BatchSizes* sz, bool scan_grids) {
  BatchImpl B;
  pgvimp_status st = prepare(count, problems, options, precision, B, scan_grids);
  if (st != PGVIMP_OK) return st;
  sz->dev = B.total();
  sz->host_in = B.in_bytes;
  sz->host_out = B.res_bytes + B.extra_bytes;
  return PGVIMP_OK;
}

pgvimp_status pgv::batch_create_staged(int count, const pgvimp_problem* problems, const pgvimp_options* options,
                                       int precision, void* arena, size_t arena_bytes, void* h_in, void* h_out,
                                       pgvimp_batch** out, bool scan_grids) {
  if (!arena || !h_in || !h_out) return fail(nullptr, PGVIMP_EINVAL, "staged batch needs arena and staging");
  return create_batch(count, problems, options, precision, arena, arena_bytes, h_in, h_out, out, scan_grids);
}

int pgv::batch_plan_status(const pgvimp_batch* b, int index) {
  const double* sc = reinterpret_cast<const double*>(b->h_out + b->off_scal) + (size_t)kScal * index;
  return (int)sc[S_STATUS];
}


static pgvimp_status finalize(pgvimp_batch* b, cudaStream_t s) {
  // The iterate may sit in buffer set 1 or 2; results are read from set 0
  // (and, with double-float storage, converted to FP64 in place).
  return launch(*b, PH_FINALIZE, 0, 0.0, s);
}
