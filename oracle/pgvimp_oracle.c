/*
 * pgvimp_oracle.c -- plain FP64 CPU oracle of P-GVIMP (arXiv 2411.03416).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  It shares no
 * code with the CUDA library.  Every routine follows the paper's definitions
 * step by step, in FP64, with no blocking, fusion or reordering:
 *
 *   prior (Alg. 1, first two lines; LTV SDE of Sec. 2.2), via Van Loan's
 *     matrix-exponential construction of the transition and the Grammian;
 *   marginals by Gaussian belief propagation on the chain (Sec. 5.1, the
 *     message equations and the belief precision);
 *   Gauss-Hermite / degree-3 quadrature of the factor moments (Sec. 4.3), the
 *     full tensor rule over all n dimensions (no reduction);
 *   gradients of the collision part in moment form (Sec. 4.1, gradients of
 *     psi_d), one factor at a time (Sec. 4.2);
 *   the KL-proximal update (Thm 1) and the largest feasible step by bisection
 *     under the KL bound and positive definiteness (App. C);
 *   statistical linear regression of the prior drift (Sec. 6.2) and the
 *     iterative outer loop (Alg. 2).
 *
 * Readings where the paper is silent or garbled (each is an option or a
 * documented default): lower Cholesky factor as sqrt(P) in the sigma points;
 * GH weights p!/(p^2 He_{p-1}(xi)^2) (the printed formula lacks the square);
 * collision factors on all N+1 states (option: interior only); psi =
 * sigma_obs*h^2 with h = max(0, eps - sdf) (option: h^2/sigma_obs^2); no dt on
 * the running cost; temperature by scaling the prior and the cost; bisection
 * starting at beta_max with a fixed number of halvings; initial mean =
 * straight-line interpolation, initial precision = prior precision; SDF values
 * node-centred with clamped bilinear / trilinear interpolation.
 */
#include "pgvimp_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ dense */

static void mm(int r, int k, int c, const double *A, const double *B, double *C) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * c + j];
      C[i * c + j] = s;
    }
}
static void tr(int r, int c, const double *A, double *At) {
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) At[j * r + i] = A[i * c + j];
}
static void symm(int n, double *A) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double s = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = s;
      A[j * n + i] = s;
    }
}
/* Gauss-Jordan elimination with partial pivoting.  Returns 0 on success. */
static int inv(int n, const double *A, double *Ainv) {
  double *M = (double *)malloc(sizeof(double) * n * 2 * n);
  if (!M) return ORA_ENOMEM;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      M[i * 2 * n + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r * 2 * n + col]) > fabs(M[piv * 2 * n + col])) piv = r;
    if (M[piv * 2 * n + col] == 0.0) { free(M); return ORA_ENOTPD; }
    if (piv != col)
      for (int j = 0; j < 2 * n; ++j) {
        double t = M[col * 2 * n + j];
        M[col * 2 * n + j] = M[piv * 2 * n + j];
        M[piv * 2 * n + j] = t;
      }
    double d = M[col * 2 * n + col];
    for (int j = 0; j < 2 * n; ++j) M[col * 2 * n + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r * 2 * n + col];
      if (f != 0.0)
        for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[col * 2 * n + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
  free(M);
  return ORA_OK;
}
/* Lower Cholesky factor A = L L^T.  Returns ORA_ENOTPD if a pivot is not > 0.
 * With rel_pivot: the smallest pivot s_j (before the square root) divided by
 * the diagonal entry A_jj it came from, or the failing pivot's ratio. */
static int chol_pivot(int n, const double *A, double *L, double *rel_pivot) {
  memset(L, 0, sizeof(double) * n * n);
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (rel_pivot) {
      double r = s / fabs(A[j * n + j]);
      if (j == 0 || r < *rel_pivot) *rel_pivot = r;
    }
    if (!(s > 0.0)) return ORA_ENOTPD;
    double d = sqrt(s);
    L[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / d;
    }
  }
  return ORA_OK;
}
static int chol(int n, const double *A, double *L) { return chol_pivot(n, A, L, NULL); }

/* Matrix exponential by scaling and squaring of the Taylor series. */
int ora_expm(int d, const double *M, double *E) {
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += fabs(M[i * d + j]);
    if (s > nrm) nrm = s;
  }
  int sq = 0;
  while (nrm > 0.5) { nrm *= 0.5; ++sq; }
  double scale = ldexp(1.0, -sq);
  double *X = (double *)malloc(sizeof(double) * d * d);
  double *term = (double *)malloc(sizeof(double) * d * d);
  double *tmp = (double *)malloc(sizeof(double) * d * d);
  if (!X || !term || !tmp) { free(X); free(term); free(tmp); return ORA_ENOMEM; }
  for (int i = 0; i < d * d; ++i) X[i] = M[i] * scale;
  for (int i = 0; i < d * d; ++i) { E[i] = 0.0; term[i] = 0.0; }
  for (int i = 0; i < d; ++i) { E[i * d + i] = 1.0; term[i * d + i] = 1.0; }
  for (int k = 1; k <= 60; ++k) {
    mm(d, d, d, term, X, tmp);
    double tn = 0.0;
    for (int i = 0; i < d * d; ++i) { term[i] = tmp[i] / k; E[i] += term[i]; tn += fabs(term[i]); }
    if (tn < 1e-300 || (k > 4 && tn < 1e-19)) break;
  }
  for (int s = 0; s < sq; ++s) {
    mm(d, d, d, E, E, tmp);
    memcpy(E, tmp, sizeof(double) * d * d);
  }
  free(X); free(term); free(tmp);
  return ORA_OK;
}

/* ------------------------------------------------------ quadrature rules */

/* Probabilists' Hermite polynomial He_k(x) by its three-term recurrence. */
static double hermite_e(int k, double x) {
  if (k == 0) return 1.0;
  double h0 = 1.0, h1 = x;
  for (int j = 1; j < k; ++j) {
    double h2 = x * h1 - j * h0;
    h0 = h1;
    h1 = h2;
  }
  return h1;
}

/* Sec. 4.3: (1) the p roots of He_p are the nodes; (2) the weights are
 * p! / (p^2 He_{p-1}(xi)^2) for the N(0,1) weight (the printed formula drops
 * the square; with it the weights sum to one).  He_p is even or odd, so its
 * roots are symmetric about 0 (0 itself is a root for odd p): the positive
 * roots are bracketed by a fine sign scan of (0, R] and refined by bisection
 * to machine precision, then mirrored. */
int ora_gh_rule(int p, double *nodes, double *weights) {
  if (p < 1 || p > 40) return ORA_EINVAL;
  int half = p / 2, found = 0;
  double pos[20];
  double R = 2.0 * sqrt((double)p) + 2.0, h = R / 400000.0;
  double xa = 0.5 * h, fa = hermite_e(p, xa);
  for (int s = 1; s <= 400000 && found < half; ++s) {
    double xb = 0.5 * h + s * h, fb = hermite_e(p, xb);
    if ((fa < 0.0) != (fb < 0.0)) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = hermite_e(p, mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else hi = mid;
      }
      pos[found++] = 0.5 * (lo + hi);
    }
    xa = xb;
    fa = fb;
  }
  if (found != half) return ORA_EINVAL;
  for (int j = 0; j < half; ++j) {
    nodes[j] = -pos[half - 1 - j];
    nodes[p - 1 - j] = pos[half - 1 - j];
  }
  if (p % 2 == 1) nodes[half] = 0.0;
  double pf = 1.0;
  for (int j = 2; j <= p; ++j) pf *= j;
  for (int j = 0; j < p; ++j) {
    double hv = hermite_e(p - 1, nodes[j]);
    weights[j] = pf / ((double)p * p * hv * hv);
  }
  return ORA_OK;
}

/* Smolyak sparse grid of level k in d dimensions (Lemma 1): the combination
 *   A(k, d) = sum_{q = max(0, k-d)}^{k-1} (-1)^{k-1-q} C(d-1, k-1-q)
 *             sum_{i_1 + ... + i_d = d + q, i_j >= 1} U^{i_1} x ... x U^{i_d}
 * of the 1-D Gauss-Hermite rules U^i with i points; exact for every
 * polynomial of total degree <= 2k - 1.  Coinciding nodes are merged (their
 * weights added).  Returns the node count; with xi == NULL only counts.
 * Written out plainly: the multi-indices in lexicographic order (an entry
 * grows only while the sum stays within d + k - 1), all tensor nodes of
 * each, a linear search for duplicates. */
static double binom(int a, int b) {
  if (b < 0 || b > a) return 0.0;
  double r = 1.0;
  for (int j = 1; j <= b; ++j) r = r * (a - b + j) / j;
  return r;
}

static int smolyak_grid(int d, int k, double *xi, double *W, int cap) {
  double nodes[11][10], wts[11][10];
  for (int p = 1; p <= k; ++p)
    if (ora_gh_rule(p, nodes[p], wts[p])) return -1;
  int count = 0;
  double *X = malloc(sizeof(double) * (size_t)cap * d), *Wt = malloc(sizeof(double) * cap);
  int *idx = malloc(sizeof(int) * d), *dig = malloc(sizeof(int) * d);
  double *pt = malloc(sizeof(double) * d);
  if (!X || !Wt || !idx || !dig || !pt) { count = -1; goto out; }
  for (int j = 0; j < d; ++j) idx[j] = 1;
  for (;;) {
    int s = 0;
    for (int j = 0; j < d; ++j) s += idx[j];
    int q = s - d;
    if (q >= (k > d ? k - d : 0) && q <= k - 1) {
      double coef = (((k - 1 - q) % 2) ? -1.0 : 1.0) * binom(d - 1, k - 1 - q);
      for (int j = 0; j < d; ++j) dig[j] = 0;
      for (;;) {
        double w = coef;
        for (int j = 0; j < d; ++j) {
          pt[j] = nodes[idx[j]][dig[j]];
          w *= wts[idx[j]][dig[j]];
        }
        int found = -1;
        for (int m = 0; m < count && found < 0; ++m) {
          int same = 1;
          for (int j = 0; j < d && same; ++j) same = (X[(size_t)m * d + j] == pt[j]);
          if (same) found = m;
        }
        if (found >= 0) {
          Wt[found] += w;
        } else {
          if (count == cap) { count = -1; goto out; }
          memcpy(X + (size_t)count * d, pt, sizeof(double) * d);
          Wt[count++] = w;
        }
        int j = d - 1;   /* next tensor node */
        while (j >= 0 && ++dig[j] == idx[j]) dig[j--] = 0;
        if (j < 0) break;
      }
    }
    /* next multi-index with sum <= d + k - 1: raise the last entry that
       can grow, reset the ones after it to 1 */
    int j = d - 1;
    for (; j >= 0; --j) {
      int rest = 0;
      for (int m = 0; m < d; ++m) rest += (m < j) ? idx[m] : 1;
      if (rest + idx[j] + 1 - 1 <= d + k - 1 && idx[j] + 1 <= k) break;
    }
    if (j < 0) break;
    ++idx[j];
    for (int m = j + 1; m < d; ++m) idx[m] = 1;
  }
  if (xi) {
    memcpy(xi, X, sizeof(double) * (size_t)count * d);
    memcpy(W, Wt, sizeof(double) * count);
  }
out:
  free(X); free(Wt); free(idx); free(dig); free(pt);
  return count;
}

static const int kSmolyakCap = 200000;

int ora_rule_size(int n, int rule, int p) {
  if (rule == ORA_RULE_DEG3) return 2 * n + 1;
  if (rule == ORA_RULE_SMOLYAK) return smolyak_grid(n, p, NULL, NULL, kSmolyakCap);
  int s = 1;
  for (int j = 0; j < n; ++j) s *= p;
  return s;
}

/* Full rule over all n dimensions.  Tensor GH: point l has digits
 * (d_0 .. d_{n-1}) of l in base p, dimension 0 most significant.
 * Degree 3 (Lemma 1's sparse family, its lowest level): {0, +-sqrt(3) e_j},
 * weights 1 - n/3 and 1/6; order: centre, then +e_0, -e_0, +e_1, ... */
int ora_rule(int n, int rule, int p, double *xi, double *W) {
  if (rule == ORA_RULE_SMOLYAK) return smolyak_grid(n, p, xi, W, kSmolyakCap) < 0 ? ORA_EINVAL : ORA_OK;
  if (rule == ORA_RULE_DEG3) {
    memset(xi, 0, sizeof(double) * (2 * n + 1) * n);
    W[0] = 1.0 - n / 3.0;
    for (int j = 0; j < n; ++j) {
      xi[(1 + 2 * j) * n + j] = sqrt(3.0);
      xi[(2 + 2 * j) * n + j] = -sqrt(3.0);
      W[1 + 2 * j] = 1.0 / 6.0;
      W[2 + 2 * j] = 1.0 / 6.0;
    }
    return ORA_OK;
  }
  double nodes[40], wts[40];
  int rc = ora_gh_rule(p, nodes, wts);
  if (rc) return rc;
  int P = ora_rule_size(n, rule, p);
  for (int l = 0; l < P; ++l) {
    int rem = l;
    double w = 1.0;
    for (int j = n - 1; j >= 0; --j) {
      int dgt = rem % p;
      rem /= p;
      xi[l * n + j] = nodes[dgt];
      w *= wts[dgt];
    }
    W[l] = w;
  }
  return ORA_OK;
}

/* ------------------------------------------------------------------ prior */

static const double *A_at(const ora_problem *pb, const double *A_ltv, int i) {
  if (A_ltv) return A_ltv + (size_t)i * pb->n * pb->n;
  return pb->A_per_step ? pb->A + (size_t)i * pb->n * pb->n : pb->A;
}
static void a_at(const ora_problem *pb, const double *a_ltv, int i, double *out) {
  int n = pb->n;
  if (a_ltv) { memcpy(out, a_ltv + (size_t)i * n, sizeof(double) * n); return; }
  if (!pb->a) { memset(out, 0, sizeof(double) * n); return; }
  memcpy(out, pb->a_per_step ? pb->a + (size_t)i * n : pb->a, sizeof(double) * n);
}
static double temp_of(const ora_problem *pb) { return pb->temperature > 0.0 ? pb->temperature : 1.0; }

/* Alg. 1, first line: per interval [t_i, t_{i+1}] with (A_i, a_i) held
 * constant, the transition Phi_i = exp(A_i dt), the Grammian
 * Q_i = int_0^dt Phi(s) B Qc B^T Phi(s)^T ds (Van Loan: expm of
 * [[-A, BQcB^T],[0, A^T]] dt gives Phi = G22^T, Q = Phi G12) and the mean
 * offset u_i = int_0^dt Phi(dt-s) a ds (expm of [[A, a],[0, 0]] dt).
 * Alg. 1, second line: prior precision K^-1 = sum_i F_i^T Q_i^-1 F_i with
 * F_i x = x_{i+1} - Phi_i x_i, plus the start and goal factors, and the
 * information vector b = K^-1 mu_bar.  Both are divided by the temperature. */
int ora_prior(const ora_problem *pb, const double *A_ltv, const double *a_ltv,
              double *Kd, double *Ko, double *b, double *Phi_out, double *Q_out, double *u_out) {
  int n = pb->n, m = pb->m, N = pb->N;
  if (n < 1 || m < 1 || N < 1 || !(pb->T > 0.0)) return ORA_EINVAL;
  double dt = pb->T / N;
  int n2 = 2 * n, n1 = n + 1;
  double *W = calloc((size_t)n * n, sizeof(double)), *BQ = calloc((size_t)n * m, sizeof(double));
  double *Bt = calloc((size_t)m * n, sizeof(double));
  double *H = calloc((size_t)n2 * n2, sizeof(double)), *EH = calloc((size_t)n2 * n2, sizeof(double));
  double *Ha = calloc((size_t)n1 * n1, sizeof(double)), *EHa = calloc((size_t)n1 * n1, sizeof(double));
  double *Phi = calloc((size_t)n * n, sizeof(double)), *G12 = calloc((size_t)n * n, sizeof(double));
  double *G22 = calloc((size_t)n * n, sizeof(double)), *Q = calloc((size_t)n * n, sizeof(double));
  double *Qi = calloc((size_t)n * n, sizeof(double)), *T1 = calloc((size_t)n * n, sizeof(double));
  double *T2 = calloc((size_t)n * n, sizeof(double)), *PhiT = calloc((size_t)n * n, sizeof(double));
  double *ai = calloc(n, sizeof(double)), *u = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
  int rc = ORA_OK;
  if (!W || !BQ || !Bt || !H || !EH || !Ha || !EHa || !Phi || !G12 || !G22 || !Q || !Qi || !T1 || !T2 ||
      !PhiT || !ai || !u || !v) { rc = ORA_ENOMEM; goto done; }
  memset(Kd, 0, sizeof(double) * (size_t)(N + 1) * n * n);
  memset(Ko, 0, sizeof(double) * (size_t)N * n * n);
  memset(b, 0, sizeof(double) * (size_t)(N + 1) * n);
  mm(n, m, m, pb->B, pb->Qc, BQ);
  tr(n, m, pb->B, Bt);
  mm(n, m, n, BQ, Bt, W);
  for (int i = 0; i < N; ++i) {
    const double *A = A_at(pb, A_ltv, i);
    a_at(pb, a_ltv, i, ai);
    memset(H, 0, sizeof(double) * n2 * n2);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        H[r * n2 + c] = -A[r * n + c] * dt;
        H[r * n2 + n + c] = W[r * n + c] * dt;
        H[(n + r) * n2 + n + c] = A[c * n + r] * dt;
      }
    if ((rc = ora_expm(n2, H, EH))) goto done;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        G12[r * n + c] = EH[r * n2 + n + c];
        G22[r * n + c] = EH[(n + r) * n2 + n + c];
      }
    tr(n, n, G22, Phi);
    mm(n, n, n, Phi, G12, Q);
    symm(n, Q);
    memset(Ha, 0, sizeof(double) * n1 * n1);
    for (int r = 0; r < n; ++r) {
      for (int c = 0; c < n; ++c) Ha[r * n1 + c] = A[r * n + c] * dt;
      Ha[r * n1 + n] = ai[r] * dt;
    }
    if ((rc = ora_expm(n1, Ha, EHa))) goto done;
    for (int r = 0; r < n; ++r) u[r] = EHa[r * n1 + n];
    if (Phi_out) memcpy(Phi_out + (size_t)i * n * n, Phi, sizeof(double) * n * n);
    if (Q_out) memcpy(Q_out + (size_t)i * n * n, Q, sizeof(double) * n * n);
    if (u_out) memcpy(u_out + (size_t)i * n, u, sizeof(double) * n);
    if ((rc = inv(n, Q, Qi))) goto done;
    symm(n, Qi);
    /* F_i^T Q^-1 F_i on (x_i, x_{i+1}) with F_i = [-Phi, I] */
    tr(n, n, Phi, PhiT);
    mm(n, n, n, PhiT, Qi, T1);              /* Phi^T Q^-1 */
    mm(n, n, n, T1, Phi, T2);               /* Phi^T Q^-1 Phi */
    for (int e = 0; e < n * n; ++e) Kd[(size_t)i * n * n + e] += T2[e];
    for (int e = 0; e < n * n; ++e) Kd[(size_t)(i + 1) * n * n + e] += Qi[e];
    mm(n, n, n, Qi, Phi, T2);               /* Q^-1 Phi */
    for (int e = 0; e < n * n; ++e) Ko[(size_t)i * n * n + e] -= T2[e];
    /* F_i^T Q^-1 u_i */
    mm(n, n, 1, T1, u, v);
    for (int r = 0; r < n; ++r) b[(size_t)i * n + r] -= v[r];
    mm(n, n, 1, Qi, u, v);
    for (int r = 0; r < n; ++r) b[(size_t)(i + 1) * n + r] += v[r];
  }
  /* start and goal factors */
  for (int side = 0; side < 2; ++side) {
    const double *K = side ? pb->KN : pb->K0, *mu = side ? pb->muN : pb->mu0;
    int at = side ? N : 0;
    if ((rc = inv(n, K, Qi))) goto done;
    symm(n, Qi);
    for (int e = 0; e < n * n; ++e) Kd[(size_t)at * n * n + e] += Qi[e];
    mm(n, n, 1, Qi, mu, v);
    for (int r = 0; r < n; ++r) b[(size_t)at * n + r] += v[r];
  }
  {
    double Th = temp_of(pb);
    for (size_t e = 0; e < (size_t)(N + 1) * n * n; ++e) Kd[e] /= Th;
    for (size_t e = 0; e < (size_t)N * n * n; ++e) Ko[e] /= Th;
    for (size_t e = 0; e < (size_t)(N + 1) * n; ++e) b[e] /= Th;
  }
done:
  free(W); free(BQ); free(Bt); free(H); free(EH); free(Ha); free(EHa); free(Phi); free(G12);
  free(G22); free(Q); free(Qi); free(T1); free(T2); free(PhiT); free(ai); free(u); free(v);
  return rc;
}

/* Block Gaussian elimination (block Thomas algorithm) for a symmetric
 * block-tridiagonal system M x = r; M_{i,i-1} = Mo[i-1]. */
int ora_block_solve(int n, int N, const double *Md, const double *Mo, const double *r, double *x) {
  size_t nn = (size_t)n * n;
  double *C = malloc(sizeof(double) * nn), *Ci = malloc(sizeof(double) * (N + 1) * nn);
  double *y = malloc(sizeof(double) * (N + 1) * n), *T = malloc(sizeof(double) * nn);
  double *MoT = malloc(sizeof(double) * nn), *T2 = malloc(sizeof(double) * nn);
  double *v = malloc(sizeof(double) * n);
  int rc = ORA_OK;
  if (!C || !Ci || !y || !T || !MoT || !T2 || !v) { rc = ORA_ENOMEM; goto done; }
  memcpy(C, Md, sizeof(double) * nn);
  memcpy(y, r, sizeof(double) * n);
  for (int i = 1; i <= N; ++i) {
    if ((rc = inv(n, C, Ci + (i - 1) * nn))) goto done;
    mm(n, n, n, Mo + (i - 1) * nn, Ci + (i - 1) * nn, T);   /* M_{i,i-1} C^-1 */
    tr(n, n, Mo + (i - 1) * nn, MoT);
    mm(n, n, n, T, MoT, T2);
    for (size_t e = 0; e < nn; ++e) C[e] = Md[i * nn + e] - T2[e];
    mm(n, n, 1, T, y + (i - 1) * n, v);
    for (int a = 0; a < n; ++a) y[i * n + a] = r[i * n + a] - v[a];
  }
  if ((rc = inv(n, C, Ci + N * nn))) goto done;
  mm(n, n, 1, Ci + N * nn, y + N * n, x + N * n);
  for (int i = N - 1; i >= 0; --i) {
    tr(n, n, Mo + i * nn, MoT);
    mm(n, n, 1, MoT, x + (i + 1) * n, v);
    for (int a = 0; a < n; ++a) v[a] = y[i * n + a] - v[a];
    mm(n, n, 1, Ci + i * nn, v, x + i * n);
  }
done:
  free(C); free(Ci); free(y); free(T); free(MoT); free(T2); free(v);
  return rc;
}

int ora_prior_mean(const ora_problem *pb, const double *Kd, const double *Ko, const double *b, double *mubar) {
  return ora_block_solve(pb->n, pb->N, Kd, Ko, b, mubar);
}

/* Initial mean (not given in the paper): positions on the straight line from
 * the start mean to the goal mean, velocities constant (goal-start)/T. */
int ora_init_mean(const ora_problem *pb, double *mu) {
  int n = pb->n, nq = n / 2, N = pb->N;
  for (int i = 0; i <= N; ++i) {
    double s = (double)i / N;
    for (int a = 0; a < nq; ++a) {
      double d = pb->muN[a] - pb->mu0[a];
      mu[i * n + a] = pb->mu0[a] + s * d;
      mu[i * n + nq + a] = d / pb->T;
    }
  }
  return ORA_OK;
}

/* -------------------------------------------------------------- marginals */

/* Sec. 5.1: Gaussian belief propagation on the chain factor graph of the
 * zero-mean Gaussian with precision Lambda.  Unary factors carry Lambda_ii,
 * pairwise factors the off-diagonal blocks.  Forward messages into x_i:
 *   F_0 = 0,  F_i = -Lambda_{i,i-1} (Lambda_{i-1,i-1} + F_{i-1})^-1 Lambda_{i-1,i};
 * backward messages:
 *   R_N = 0,  R_i = -Lambda_{i,i+1} (Lambda_{i+1,i+1} + R_{i+1})^-1 Lambda_{i+1,i};
 * belief precision Lambda_b_i = Lambda_ii + F_i + R_i, marginal Sigma_ii =
 * Lambda_b_i^-1; the pairwise belief of (x_i, x_{i+1}) gives Sigma_{i+1,i}.
 * log det Lambda = sum_i log det(Lambda_ii + F_i) (Schur complements); the
 * matrix is positive definite iff every such block is. */
int ora_marginals(int n, int N, const double *Ld, const double *Lo, double *Sd, double *So, double *logdet) {
  return ora_marginals_pivot(n, N, Ld, Lo, Sd, So, logdet, NULL);
}

int ora_marginals_pivot(int n, int N, const double *Ld, const double *Lo, double *Sd, double *So,
                        double *logdet, double *rel_pivot) {
  size_t nn = (size_t)n * n;
  double piv_min = INFINITY;
  int n2 = 2 * n;
  double *F = calloc((N + 1) * nn, sizeof(double)), *R = calloc((N + 1) * nn, sizeof(double));
  double *P = malloc(sizeof(double) * nn), *Pi = malloc(sizeof(double) * nn), *L = malloc(sizeof(double) * nn);
  double *T = malloc(sizeof(double) * nn), *OT = malloc(sizeof(double) * nn);
  double *J = malloc(sizeof(double) * n2 * n2), *Ji = malloc(sizeof(double) * n2 * n2);
  int rc = ORA_OK;
  double ld = 0.0;
  if (!F || !R || !P || !Pi || !L || !T || !OT || !J || !Ji) { rc = ORA_ENOMEM; goto done; }
  for (int i = 0; i <= N; ++i) {
    for (size_t e = 0; e < nn; ++e) P[e] = Ld[i * nn + e] + F[i * nn + e];
    double piv;
    rc = chol_pivot(n, P, L, &piv);
    if (piv < piv_min) piv_min = piv;
    if (rc) goto done;
    for (int a = 0; a < n; ++a) ld += 2.0 * log(L[a * n + a]);
    if (i == N) break;
    if ((rc = inv(n, P, Pi))) goto done;
    mm(n, n, n, Lo + i * nn, Pi, T);           /* Lambda_{i+1,i} P^-1 */
    tr(n, n, Lo + i * nn, OT);                 /* Lambda_{i,i+1} */
    mm(n, n, n, T, OT, F + (i + 1) * nn);
    for (size_t e = 0; e < nn; ++e) F[(i + 1) * nn + e] = -F[(i + 1) * nn + e];
    symm(n, F + (i + 1) * nn);
  }
  for (int i = N - 1; i >= 0; --i) {
    for (size_t e = 0; e < nn; ++e) P[e] = Ld[(i + 1) * nn + e] + R[(i + 1) * nn + e];
    if ((rc = inv(n, P, Pi))) goto done;
    tr(n, n, Lo + i * nn, OT);                 /* Lambda_{i,i+1} */
    mm(n, n, n, OT, Pi, T);
    mm(n, n, n, T, Lo + i * nn, R + i * nn);
    for (size_t e = 0; e < nn; ++e) R[i * nn + e] = -R[i * nn + e];
    symm(n, R + i * nn);
  }
  for (int i = 0; i <= N; ++i) {
    for (size_t e = 0; e < nn; ++e) P[e] = Ld[i * nn + e] + F[i * nn + e] + R[i * nn + e];
    if ((rc = inv(n, P, Sd + i * nn))) goto done;
    symm(n, Sd + i * nn);
  }
  for (int i = 0; i < N; ++i) {
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        J[a * n2 + c] = Ld[i * nn + a * n + c] + F[i * nn + a * n + c];
        J[a * n2 + n + c] = Lo[i * nn + c * n + a];
        J[(n + a) * n2 + c] = Lo[i * nn + a * n + c];
        J[(n + a) * n2 + n + c] = Ld[(i + 1) * nn + a * n + c] + R[(i + 1) * nn + a * n + c];
      }
    if ((rc = inv(n2, J, Ji))) goto done;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) So[i * nn + a * n + c] = Ji[(n + a) * n2 + c];
  }
done:
  if (logdet) *logdet = ld;
  if (rel_pivot) *rel_pivot = piv_min;
  free(F); free(R); free(P); free(Pi); free(L); free(T); free(OT); free(J); free(Ji);
  return rc;
}

/* ------------------------------------------------------- cost and moments */

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Signed distance at a position: node-centred grid values at
 * origin + index*cell, coordinates clamped to the grid, bilinear (2-D,
 * sdf_nz <= 1) or trilinear (3-D) interpolation in FP64 of FP32 values. */
double ora_sdf(const ora_problem *pb, const double *pos) {
  int nx = pb->sdf_nx, ny = pb->sdf_ny, nz = pb->sdf_nz;
  double u[3];
  int i0[3], dims = (nz > 1) ? 3 : 2;
  int sz[3] = {nx, ny, nz};
  double f[3];
  for (int d = 0; d < dims; ++d) {
    u[d] = clampd((pos[d] - pb->sdf_origin[d]) / pb->sdf_cell, 0.0, (double)(sz[d] - 1));
    i0[d] = (int)floor(u[d]);
    if (i0[d] > sz[d] - 2) i0[d] = sz[d] - 2;
    f[d] = u[d] - i0[d];
  }
  if (dims == 2) {
    const float *g = pb->sdf;
    double v00 = g[(size_t)i0[1] * nx + i0[0]], v10 = g[(size_t)i0[1] * nx + i0[0] + 1];
    double v01 = g[(size_t)(i0[1] + 1) * nx + i0[0]], v11 = g[(size_t)(i0[1] + 1) * nx + i0[0] + 1];
    return (1 - f[0]) * (1 - f[1]) * v00 + f[0] * (1 - f[1]) * v10 + (1 - f[0]) * f[1] * v01 + f[0] * f[1] * v11;
  }
  double s = 0.0;
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
    s += w * pb->sdf[((size_t)(i0[2] + dz) * ny + (i0[1] + dy)) * nx + (i0[0] + dx)];
  }
  return s;
}

/* Forward kinematics of a revolute chain in standard Denavit-Hartenberg form:
 * T_j = T_{j-1} Rz(theta_j) Tz(d_j) Tx(a_j) Rx(alpha_j), theta_j = q_j + theta0_j.
 * A sphere on link j sits at a fixed offset in the frame T_{j-1} Rz(theta_j). */
int ora_arm_fk(const ora_problem *pb, const double *q, double *centres) {
  double T[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1}, R[16], Z[16], X[16], tmp[16];
  for (int j = 0; j < pb->arm_dof; ++j) {
    double a = pb->dh[4 * j], al = pb->dh[4 * j + 1], d = pb->dh[4 * j + 2], th = q[j] + pb->dh[4 * j + 3];
    double c = cos(th), s = sin(th), ca = cos(al), sa = sin(al);
    double Rz[16] = {c, -s, 0, 0, s, c, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    mm(4, 4, 4, T, Rz, R);
    for (int k = 0; k < pb->n_spheres; ++k) {
      if (pb->sphere_link[k] != j) continue;
      const double *o = pb->sphere_off + 3 * k;
      for (int r = 0; r < 3; ++r)
        centres[3 * k + r] = R[4 * r] * o[0] + R[4 * r + 1] * o[1] + R[4 * r + 2] * o[2] + R[4 * r + 3];
    }
    double Tz[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, d, 0, 0, 0, 1};
    double Tx[16] = {1, 0, 0, a, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double Rx[16] = {1, 0, 0, 0, 0, ca, -sa, 0, 0, sa, ca, 0, 0, 0, 0, 1};
    mm(4, 4, 4, R, Tz, Z);
    mm(4, 4, 4, Z, Tx, X);
    mm(4, 4, 4, X, Rx, tmp);
    memcpy(T, tmp, sizeof(T));
  }
  return ORA_OK;
}

static double hinge_cost(const ora_problem *pb, double h) {
  if (h <= 0.0) return 0.0;
  return pb->psi_form == 1 ? h * h / (pb->sigma_obs * pb->sigma_obs) : pb->sigma_obs * h * h;
}

/* Collision factor psi_i(x_i) (Sec. 4.1): hinge of the signed distance,
 * h = max(0, eps - sdf), weighted by Sigma_obs; for the arm summed over the
 * body spheres with margin eps + r_s.  Divided by the temperature. */
double ora_psi(const ora_problem *pb, int i, const double *x) {
  if (pb->factor_set == 1 && (i == 0 || i == pb->N)) return 0.0;
  double v = 0.0;
  switch (pb->cost_kind) {
    case ORA_COST_NONE: v = 0.0; break;
    case ORA_COST_POINT2D:
    case ORA_COST_POINT3D: v = hinge_cost(pb, pb->eps - ora_sdf(pb, x)); break;
    case ORA_COST_ARM: {
      double *c = malloc(sizeof(double) * 3 * pb->n_spheres);
      if (!c) return NAN;
      ora_arm_fk(pb, x, c);
      for (int k = 0; k < pb->n_spheres; ++k)
        v += hinge_cost(pb, pb->eps + pb->sphere_r[k] - ora_sdf(pb, c + 3 * k));
      free(c);
      break;
    }
    case ORA_COST_QUADRATIC: {
      int n = pb->n;
      const double *c = pb->quad_c + (size_t)i * n, *W = pb->quad_W + (size_t)i * n * n;
      for (int a = 0; a < n; ++a)
        for (int b2 = 0; b2 < n; ++b2) v += 0.5 * (x[a] - c[a]) * W[a * n + b2] * (x[b2] - c[b2]);
      break;
    }
    default: return NAN;
  }
  return v / temp_of(pb);
}

/* Sec. 4.3 applied to the three expectations of Sec. 4.1:
 * S0 = E[psi], S1 = E[(x-mu) psi], S2 = E[(x-mu)(x-mu)^T psi] under
 * N(mu_i, Sigma_ii), with sigma points x_l = mu_i + L xi_l, L = chol(Sigma_ii). */
int ora_quad_moments(const ora_problem *pb, const ora_options *op, int i, const double *mu_i,
                     const double *Sig_ii, double *S0, double *S1, double *S2) {
  int n = pb->n, P = ora_rule_size(n, op->rule, op->gh_p), rc;
  double *xi = malloc(sizeof(double) * (size_t)P * n), *W = malloc(sizeof(double) * P);
  double *L = malloc(sizeof(double) * n * n), *x = malloc(sizeof(double) * n), *d = malloc(sizeof(double) * n);
  if (!xi || !W || !L || !x || !d) { rc = ORA_ENOMEM; goto done; }
  if ((rc = ora_rule(n, op->rule, op->gh_p, xi, W))) goto done;
  if ((rc = chol(n, Sig_ii, L))) goto done;
  *S0 = 0.0;
  memset(S1, 0, sizeof(double) * n);
  memset(S2, 0, sizeof(double) * n * n);
  for (int l = 0; l < P; ++l) {
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += L[a * n + c] * xi[(size_t)l * n + c];
      d[a] = s;
      x[a] = mu_i[a] + s;
    }
    double w = W[l] * ora_psi(pb, i, x);
    *S0 += w;
    for (int a = 0; a < n; ++a) {
      S1[a] += w * d[a];
      for (int c = 0; c < n; ++c) S2[a * n + c] += w * d[a] * d[c];
    }
  }
done:
  free(xi); free(W); free(L); free(x); free(d);
  return rc;
}

/* Gradients of psi_d in moment form (Sec. 4.1), for one factor (Sec. 4.2):
 * g = Sigma^-1 S1;  G = -1/2 Sigma^-1 S0 + 1/2 Sigma^-1 S2 Sigma^-1. */
int ora_gradients(int n, const double *Sig_ii, double S0, const double *S1, const double *S2,
                  double *g, double *G) {
  double *Si = malloc(sizeof(double) * n * n), *T = malloc(sizeof(double) * n * n);
  int rc;
  if (!Si || !T) { rc = ORA_ENOMEM; goto done; }
  if ((rc = inv(n, Sig_ii, Si))) goto done;
  mm(n, n, 1, Si, S1, g);
  mm(n, n, n, Si, S2, T);
  mm(n, n, n, T, Si, G);
  for (int e = 0; e < n * n; ++e) G[e] = 0.5 * G[e] - 0.5 * S0 * Si[e];
  symm(n, G);
done:
  free(Si); free(T);
  return rc;
}

/* ------------------------------------------------------------ the update */

/* y = Lambda x for a block-tridiagonal symmetric Lambda. */
static void bt_matvec(int n, int N, const double *Ld, const double *Lo, const double *x, double *y) {
  size_t nn = (size_t)n * n;
  for (int i = 0; i <= N; ++i)
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += Ld[i * nn + a * n + c] * x[i * n + c];
      if (i > 0)
        for (int c = 0; c < n; ++c) s += Lo[(i - 1) * nn + a * n + c] * x[(i - 1) * n + c];
      if (i < N)
        for (int c = 0; c < n; ++c) s += Lo[i * nn + c * n + a] * x[(i + 1) * n + c];
      y[i * n + a] = s;
    }
}
/* tr(Lambda Sigma) over the block-tridiagonal support of Lambda. */
static double bt_trace(int n, int N, const double *Ld, const double *Lo, const double *Sd, const double *So) {
  size_t nn = (size_t)n * n;
  double t = 0.0;
  for (int i = 0; i <= N; ++i)
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) t += Ld[i * nn + a * n + c] * Sd[i * nn + c * n + a];
  for (int i = 0; i < N; ++i)
    for (size_t e = 0; e < nn; ++e) t += 2.0 * Lo[i * nn + e] * So[i * nn + e];
  return t;
}

/* Thm 1 at step size beta (update ORA_UPDATE_PROX):
 *   (K^-1 + Lambda_k/beta) mu' = -g + K^-1 mu_bar + Lambda_k mu_k / beta
 *   Lambda' = beta/(beta+1) (2G + K^-1 + Lambda_k/beta)
 * (G is block-diagonal, so it only enters the diagonal blocks).
 *
 * NGD at step size beta (update ORA_UPDATE_NGD, Sec. 3.1(d)): the natural-
 * gradient step delta theta = beta G(theta)^-1 grad L, with the Fisher matrix
 * G(theta).  For a Gaussian in natural parameters eta = (Lambda mu, -Lambda/2)
 * the Fisher matrix is the Jacobian of the expectation parameters
 * m = (mu, mu mu^T + Sigma) with respect to eta, so the step is
 * eta' = eta - beta grad_m J, J = -L = E[psi_d] + psi_e up to a constant.
 * With grad_Sigma E[psi_d] = G, grad_mu E[psi_d] = g, and for psi_e (the
 * prior and entropy part) grad_Sigma = K^-1/2 - Lambda/2, grad_mu =
 * K^-1 mu - K^-1 mu_bar:
 *   grad_{m2} J = G + K^-1/2 - Lambda_k/2,
 *   grad_{m1} J = grad_mu J - 2 (grad_{m2} J) mu_k = g - b - 2 G mu_k + Lambda_k mu_k,
 * hence
 *   Lambda'     = (1 - beta) Lambda_k + beta (K^-1 + 2G),
 *   Lambda' mu' = (1 - beta) Lambda_k mu_k + beta (b - g + 2 G mu_k),   b = K^-1 mu_bar.
 *
 * Then, for either update, the marginals of Lambda' (which also decide
 * Lambda' > 0) and the Gaussian
 * KL(q'||q_k) = 1/2 [tr(Lambda_k Sigma') + dmu^T Lambda_k dmu - D
 *                    + log det Lambda' - log det Lambda_k],
 * with the trace term written as tr((Lambda_k - Lambda') Sigma') + D.
 * Returns ORA_ENOTPD (kl = +inf) when Lambda' is not positive definite. */
int ora_trial_ex(const ora_problem *pb, int update, double beta, const double *Kd, const double *Ko,
                 const double *b, const double *mu, const double *Ld, const double *Lo, double logdet_k,
                 const double *g, const double *G,
                 double *mu_new, double *Ld_new, double *Lo_new, double *Sd_new, double *So_new,
                 double *logdet_new, double *kl, double *rel_pivot) {
  int n = pb->n, N = pb->N, D = n * (N + 1);
  size_t nn = (size_t)n * n;
  double *Md = malloc(sizeof(double) * (N + 1) * nn), *Mo = malloc(sizeof(double) * (N > 0 ? N : 1) * nn);
  double *r = malloc(sizeof(double) * D), *Lm = malloc(sizeof(double) * D), *dm = malloc(sizeof(double) * D);
  int rc = ORA_OK;
  *kl = INFINITY;
  if (rel_pivot) *rel_pivot = NAN;
  if (!Md || !Mo || !r || !Lm || !dm) { rc = ORA_ENOMEM; goto done; }
  if (update == ORA_UPDATE_NGD) {
    for (int i = 0; i <= N; ++i)
      for (size_t e = 0; e < nn; ++e)
        Ld_new[i * nn + e] = (1.0 - beta) * Ld[i * nn + e] + beta * (Kd[i * nn + e] + 2.0 * G[i * nn + e]);
    for (int i = 0; i <= N; ++i) symm(n, Ld_new + i * nn);
    for (int i = 0; i < N; ++i)
      for (size_t e = 0; e < nn; ++e) Lo_new[i * nn + e] = (1.0 - beta) * Lo[i * nn + e] + beta * Ko[i * nn + e];
    bt_matvec(n, N, Ld, Lo, mu, Lm);
    for (int i = 0; i <= N; ++i)
      for (int a = 0; a < n; ++a) {
        double Gm = 0.0;
        for (int c = 0; c < n; ++c) Gm += G[i * nn + a * n + c] * mu[i * n + c];
        r[i * n + a] = (1.0 - beta) * Lm[i * n + a] + beta * (b[i * n + a] - g[i * n + a] + 2.0 * Gm);
      }
    if ((rc = ora_block_solve(n, N, Ld_new, Lo_new, r, mu_new))) goto done;
  } else {
    double c = beta / (beta + 1.0);
    for (int i = 0; i <= N; ++i)
      for (size_t e = 0; e < nn; ++e) {
        Ld_new[i * nn + e] = c * (2.0 * G[i * nn + e] + Kd[i * nn + e] + Ld[i * nn + e] / beta);
        Md[i * nn + e] = Kd[i * nn + e] + Ld[i * nn + e] / beta;
      }
    for (int i = 0; i <= N; ++i) symm(n, Ld_new + i * nn);
    for (int i = 0; i < N; ++i)
      for (size_t e = 0; e < nn; ++e) {
        Lo_new[i * nn + e] = c * (Ko[i * nn + e] + Lo[i * nn + e] / beta);
        Mo[i * nn + e] = Ko[i * nn + e] + Lo[i * nn + e] / beta;
      }
    bt_matvec(n, N, Ld, Lo, mu, Lm);
    for (int e = 0; e < D; ++e) r[e] = -g[e] + b[e] + Lm[e] / beta;
    if ((rc = ora_block_solve(n, N, Md, Mo, r, mu_new))) goto done;
  }
  if ((rc = ora_marginals_pivot(n, N, Ld_new, Lo_new, Sd_new, So_new, logdet_new, rel_pivot))) goto done;
  for (int e = 0; e < D; ++e) dm[e] = mu_new[e] - mu[e];
  bt_matvec(n, N, Ld, Lo, dm, Lm);
  double quad = 0.0;
  for (int e = 0; e < D; ++e) quad += dm[e] * Lm[e];
  /* tr(Lambda_k Sigma') - D = tr((Lambda_k - Lambda') Sigma') exactly; the
   * right side avoids cancelling D against a trace of very large terms.  The
   * difference Lambda_k - Lambda' reuses the Md/Mo buffers. */
  for (size_t e = 0; e < (size_t)(N + 1) * nn; ++e) Md[e] = Ld[e] - Ld_new[e];
  for (size_t e = 0; e < (size_t)N * nn; ++e) Mo[e] = Lo[e] - Lo_new[e];
  *kl = 0.5 * (bt_trace(n, N, Md, Mo, Sd_new, So_new) + quad + *logdet_new - logdet_k);
done:
  free(Md); free(Mo); free(r); free(Lm); free(dm);
  return rc;
}

int ora_trial(const ora_problem *pb, double beta, const double *Kd, const double *Ko, const double *b,
              const double *mu, const double *Ld, const double *Lo, double logdet_k,
              const double *g, const double *G,
              double *mu_new, double *Ld_new, double *Lo_new, double *Sd_new, double *So_new,
              double *logdet_new, double *kl) {
  return ora_trial_ex(pb, ORA_UPDATE_PROX, beta, Kd, Ko, b, mu, Ld, Lo, logdet_k, g, G, mu_new, Ld_new,
                      Lo_new, Sd_new, So_new, logdet_new, kl, NULL);
}

/* One proximal iteration of Alg. 1: factor expectations (Sec. 4.3) and the
 * gradients mapped back to the joint level (Sec. 4.2: the selection M_i puts
 * each factor's g_i, G_i at state i), then the largest step by bisection
 * (App. C): try beta_max; if infeasible, halve the bracket [0, beta_max]
 * max_bisect times, keeping the feasible side; beta = 0 means no move.
 * Feasible: Lambda' > 0 and KL(q'||q_k) <= eps.  The log records the costs of
 * the iterate q_k the gradients were taken at. */
int ora_step(const ora_problem *pb, const ora_options *op, int k,
             const double *Kd, const double *Ko, const double *b, const double *mubar,
             double *mu, double *Ld, double *Lo, double *Sd, double *So, double *logdet,
             ora_iter_log *out_log) {
  int n = pb->n, N = pb->N, D = n * (N + 1);
  size_t nn = (size_t)n * n, dsz = (size_t)(N + 1) * nn, osz = (size_t)N * nn;
  double *g = malloc(sizeof(double) * D), *G = malloc(sizeof(double) * dsz);
  double *S1 = malloc(sizeof(double) * n), *S2 = malloc(sizeof(double) * nn);
  double *tm = malloc(sizeof(double) * D), *tLd = malloc(sizeof(double) * dsz), *tLo = malloc(sizeof(double) * (osz ? osz : 1));
  double *tSd = malloc(sizeof(double) * dsz), *tSo = malloc(sizeof(double) * (osz ? osz : 1));
  double *bm = malloc(sizeof(double) * D), *bLd = malloc(sizeof(double) * dsz), *bLo = malloc(sizeof(double) * (osz ? osz : 1));
  double *bSd = malloc(sizeof(double) * dsz), *bSo = malloc(sizeof(double) * (osz ? osz : 1));
  double *dm = malloc(sizeof(double) * D), *Km = malloc(sizeof(double) * D);
  int rc = ORA_OK;
  ora_iter_log lg;
  memset(&lg, 0, sizeof(lg));
  if (!g || !G || !S1 || !S2 || !tm || !tLd || !tLo || !tSd || !tSo || !bm || !bLd || !bLo || !bSd || !bSo || !dm || !Km) {
    rc = ORA_ENOMEM;
    goto done;
  }
  double coll = 0.0;
  for (int i = 0; i <= N; ++i) {
    double S0;
    if ((rc = ora_quad_moments(pb, op, i, mu + i * n, Sd + i * nn, &S0, S1, S2))) goto done;
    coll += S0;
    if ((rc = ora_gradients(n, Sd + i * nn, S0, S1, S2, g + i * n, G + i * nn))) goto done;
  }
  for (int e = 0; e < D; ++e) dm[e] = mu[e] - mubar[e];
  bt_matvec(n, N, Kd, Ko, dm, Km);
  double pq = 0.0;
  for (int e = 0; e < D; ++e) pq += dm[e] * Km[e];
  lg.prior_cost = 0.5 * (bt_trace(n, N, Kd, Ko, Sd, So) + pq);
  lg.collision_cost = coll;
  lg.entropy = 0.5 * (D * (1.0 + log(2.0 * 3.14159265358979323846)) - *logdet);
  lg.kl_margin = INFINITY;

  double best_beta = 0.0, best_kl = 0.0, best_ld = 0.0;
  int have = 0;
  double eps = op->kl_eps;
  lg.pd_margin = INFINITY;
  /* One trial of the own search: feasible = Lambda' > 0 and KL <= eps.  The
   * trial is recorded (beta, KL, smallest relative pivot, decisions). */
#define TRY(beta_, feas_)                                                                              \
  do {                                                                                                 \
    double kl_, ld_, piv_;                                                                             \
    int trc_ = ora_trial_ex(pb, op->update, (beta_), Kd, Ko, b, mu, Ld, Lo, *logdet, g, G, tm, tLd,    \
                            tLo, tSd, tSo, &ld_, &kl_, &piv_);                                         \
    if (trc_ == ORA_ENOMEM) { rc = trc_; goto done; }                                                  \
    lg.trials++;                                                                                       \
    (feas_) = (trc_ == ORA_OK) && (kl_ <= eps);                                                        \
    if (trc_ == ORA_OK && isfinite(eps) && eps > 0) {                                                  \
      double mg_ = fabs(kl_ - eps) / eps;                                                              \
      if (mg_ < lg.kl_margin) lg.kl_margin = mg_;                                                      \
    }                                                                                                  \
    if (fabs(piv_) < lg.pd_margin) lg.pd_margin = fabs(piv_);                                          \
    if (op->trials_out && op->trials_n && *op->trials_n < op->trials_cap) {                            \
      ora_trial_rec *t_ = op->trials_out + (*op->trials_n)++;                                          \
      t_->iter = k;                                                                                    \
      t_->pd = (trc_ == ORA_OK);                                                                       \
      t_->feasible = (feas_);                                                                          \
      t_->pad = 0;                                                                                     \
      t_->beta = (beta_);                                                                              \
      t_->kl = (trc_ == ORA_OK) ? kl_ : INFINITY;                                                      \
      t_->rel_pivot = piv_;                                                                            \
    }                                                                                                  \
    if (feas_) {                                                                                       \
      best_beta = (beta_); best_kl = kl_; best_ld = ld_; have = 1;                                     \
      memcpy(bm, tm, sizeof(double) * D); memcpy(bLd, tLd, sizeof(double) * dsz);                     \
      memcpy(bLo, tLo, sizeof(double) * osz); memcpy(bSd, tSd, sizeof(double) * dsz);                 \
      memcpy(bSo, tSo, sizeof(double) * osz);                                                          \
    }                                                                                                  \
  } while (0)
  int feas = 0;
  TRY(op->beta_max, feas);
  if (!feas) {
    double lo = 0.0, hi = op->beta_max;
    for (int t = 0; t < op->max_bisect; ++t) {
      double mid = 0.5 * (lo + hi);
      TRY(mid, feas);
      if (feas) lo = mid; else hi = mid;
    }
  }
#undef TRY
  lg.beta_own = have ? best_beta : 0.0;
  if (op->replay_beta && op->replay_beta[k] != lg.beta_own) {
    /* replay: the step decided elsewhere is taken whenever Lambda'(beta) is
     * positive definite; its KL is recorded, not enforced */
    double bt = op->replay_beta[k];
    lg.replayed = 1;
    have = 0;
    if (bt > 0.0) {
      double kl_, ld_;
      int trc_ = ora_trial_ex(pb, op->update, bt, Kd, Ko, b, mu, Ld, Lo, *logdet, g, G, bm, bLd, bLo, bSd,
                              bSo, &ld_, &kl_, NULL);
      if (trc_ == ORA_ENOMEM) { rc = trc_; goto done; }
      if (trc_ == ORA_OK) {
        best_beta = bt; best_kl = kl_; best_ld = ld_; have = 1;
      }
    }
  }
  if (have) {
    memcpy(mu, bm, sizeof(double) * D);
    memcpy(Ld, bLd, sizeof(double) * dsz);
    memcpy(Lo, bLo, sizeof(double) * osz);
    memcpy(Sd, bSd, sizeof(double) * dsz);
    memcpy(So, bSo, sizeof(double) * osz);
    *logdet = best_ld;
    lg.beta = best_beta;
    lg.kl = best_kl;
    lg.accepted = 1;
  }
done:
  if (out_log) *out_log = lg;
  free(g); free(G); free(S1); free(S2); free(tm); free(tLd); free(tLo); free(tSd); free(tSo);
  free(bm); free(bLd); free(bLo); free(bSd); free(bSo); free(dm); free(Km);
  return rc;
}

/* The problem at global iteration k: the problem itself, or, from the
 * temperature switch on, a copy with T-hat = temperature_high. */
static int hot_phase(const ora_options *op, int k) {
  return op->switch_iter > 0 && op->temperature_high > 0.0 && k >= op->switch_iter;
}

/* Alg. 1: prior, initial iterate (init != 0) or the given (mu, Lambda), its
 * marginals, then op->iters proximal iterations.  At the temperature switch
 * the prior (K^-1, b) is rebuilt at the high temperature and the cost is
 * divided by it from then on. */
int ora_plan(const ora_problem *pb, const ora_options *op, int init, double *mu, double *Ld,
             double *Lo, double *Sd, double *So, ora_iter_log *logs) {
  int n = pb->n, N = pb->N;
  size_t nn = (size_t)n * n;
  double *Kd = malloc(sizeof(double) * (N + 1) * nn), *Ko = malloc(sizeof(double) * N * nn);
  double *b = malloc(sizeof(double) * (N + 1) * n), *mubar = malloc(sizeof(double) * (N + 1) * n);
  int rc = ORA_OK;
  double logdet;
  if (!Kd || !Ko || !b || !mubar) { rc = ORA_ENOMEM; goto done; }
  if ((rc = ora_prior(pb, NULL, NULL, Kd, Ko, b, NULL, NULL, NULL))) goto done;
  if ((rc = ora_prior_mean(pb, Kd, Ko, b, mubar))) goto done;
  if (init) {
    ora_init_mean(pb, mu);
    if (op->init_kind == 1) {
      memset(Ld, 0, sizeof(double) * (N + 1) * nn);
      memset(Lo, 0, sizeof(double) * N * nn);
      for (int i = 0; i <= N; ++i)
        for (int a = 0; a < n; ++a) Ld[i * nn + a * n + a] = op->init_scale;
    } else {
      memcpy(Ld, Kd, sizeof(double) * (N + 1) * nn);
      memcpy(Lo, Ko, sizeof(double) * N * nn);
    }
  }
  if ((rc = ora_marginals(n, N, Ld, Lo, Sd, So, &logdet))) goto done;
  {
    ora_problem hot = *pb;
    hot.temperature = op->temperature_high;
    const ora_problem *cur = pb;
    for (int k = 0; k < op->iters; ++k) {
      if (hot_phase(op, k) && cur == pb) {
        cur = &hot;
        if ((rc = ora_prior(cur, NULL, NULL, Kd, Ko, b, NULL, NULL, NULL))) goto done;
        if ((rc = ora_prior_mean(cur, Kd, Ko, b, mubar))) goto done;
      }
      if ((rc = ora_step(cur, op, k, Kd, Ko, b, mubar, mu, Ld, Lo, Sd, So, &logdet, logs ? logs + k : NULL)))
        goto done;
    }
  }
done:
  free(Kd); free(Ko); free(b); free(mubar);
  return rc;
}

/* ---------------------------------------------------------- SLR, Alg. 2 */

/* Prior drift f_0(x) = f(x, u = 0).  Planar quadrotor, eq. (planar_quad):
 * x = (p_x, p_z, phi, v_x, v_z, phidot). */
int ora_drift(const ora_problem *pb, const double *x, double *f) {
  int n = pb->n;
  if (pb->dyn_kind == ORA_DYN_PLANAR_QUAD) {
    double g = pb->dyn_params[3], phi = x[2], vx = x[3], vz = x[4], w = x[5];
    f[0] = vx * cos(phi) - vz * sin(phi);
    f[1] = vx * sin(phi) + vz * cos(phi);
    f[2] = w;
    f[3] = vz * w - g * sin(phi);
    f[4] = -vx * w - g * cos(phi);
    f[5] = 0.0;
    return ORA_OK;
  }
  if (pb->dyn_kind == ORA_DYN_AFFINE_TEST) {
    for (int a = 0; a < n; ++a) {
      double s = pb->dyn_c ? pb->dyn_c[a] : 0.0;
      for (int c = 0; c < n; ++c) s += pb->dyn_F[a * n + c] * x[c];
      f[a] = s;
    }
    return ORA_OK;
  }
  return ORA_EINVAL;
}

/* Sec. 6.2: per interval i = 0..N-1, E[f], E[X], P_yx = E[(f - Ef)(X - EX)^T],
 * P_xx = E[(X - EX)(X - EX)^T] by quadrature over N(xbar_i, Sbar_i);
 * A_i = P_yx P_xx^-1, a_i = E f - A_i E X. */
int ora_slr(const ora_problem *pb, const ora_options *op, const double *xbar, const double *Sbar,
            double *A_out, double *a_out) {
  int n = pb->n, N = pb->N, P = ora_rule_size(n, op->rule, op->gh_p), rc;
  size_t nn = (size_t)n * n;
  double *xi = malloc(sizeof(double) * (size_t)P * n), *W = malloc(sizeof(double) * P);
  double *X = malloc(sizeof(double) * (size_t)P * n), *F = malloc(sizeof(double) * (size_t)P * n);
  double *L = malloc(sizeof(double) * nn), *Pyx = malloc(sizeof(double) * nn), *Pxx = malloc(sizeof(double) * nn);
  double *Pxi = malloc(sizeof(double) * nn), *Ef = malloc(sizeof(double) * n), *Ex = malloc(sizeof(double) * n);
  if (!xi || !W || !X || !F || !L || !Pyx || !Pxx || !Pxi || !Ef || !Ex) { rc = ORA_ENOMEM; goto done; }
  if ((rc = ora_rule(n, op->rule, op->gh_p, xi, W))) goto done;
  for (int i = 0; i < N; ++i) {
    if ((rc = chol(n, Sbar + i * nn, L))) goto done;
    memset(Ef, 0, sizeof(double) * n);
    memset(Ex, 0, sizeof(double) * n);
    for (int l = 0; l < P; ++l) {
      for (int a = 0; a < n; ++a) {
        double s = xbar[i * n + a];
        for (int c = 0; c < n; ++c) s += L[a * n + c] * xi[(size_t)l * n + c];
        X[(size_t)l * n + a] = s;
      }
      if ((rc = ora_drift(pb, X + (size_t)l * n, F + (size_t)l * n))) goto done;
      for (int a = 0; a < n; ++a) {
        Ef[a] += W[l] * F[(size_t)l * n + a];
        Ex[a] += W[l] * X[(size_t)l * n + a];
      }
    }
    memset(Pyx, 0, sizeof(double) * nn);
    memset(Pxx, 0, sizeof(double) * nn);
    for (int l = 0; l < P; ++l)
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
          double dxc = X[(size_t)l * n + c] - Ex[c];
          Pyx[a * n + c] += W[l] * (F[(size_t)l * n + a] - Ef[a]) * dxc;
          Pxx[a * n + c] += W[l] * (X[(size_t)l * n + a] - Ex[a]) * dxc;
        }
    if ((rc = inv(n, Pxx, Pxi))) goto done;
    mm(n, n, n, Pyx, Pxi, A_out + i * nn);
    for (int a = 0; a < n; ++a) {
      double s = Ef[a];
      for (int c = 0; c < n; ++c) s -= A_out[i * nn + a * n + c] * Ex[c];
      a_out[i * n + a] = s;
    }
  }
done:
  free(xi); free(W); free(X); free(F); free(L); free(Pyx); free(Pxx); free(Pxi); free(Ef); free(Ex);
  return rc;
}

/* Alg. 2 with the outer index j = 0..J-1: linearise the prior drift by SLR
 * around the nominal (j = 0: the straight line with covariance K0 at every
 * state; then the previous solution's mean and marginal covariances), rebuild
 * the prior of the linearised system, run Alg. 1 warm-started from the
 * previous (mu, Lambda) (Lambda = K^-1 of the first linearisation at j = 0),
 * and record ||xbar^{j+1} - xbar^j||_2. */
int ora_plan_slr(const ora_problem *pb, const ora_options *op, double *mu, double *Ld, double *Lo,
                 double *Sd, double *So, ora_iter_log *logs, double *slr_norms) {
  int n = pb->n, N = pb->N, D = n * (N + 1);
  size_t nn = (size_t)n * n;
  double *xbar = malloc(sizeof(double) * D), *Sbar = malloc(sizeof(double) * (N + 1) * nn);
  double *Al = malloc(sizeof(double) * N * nn), *al = malloc(sizeof(double) * N * n);
  double *Kd = malloc(sizeof(double) * (N + 1) * nn), *Ko = malloc(sizeof(double) * N * nn);
  double *b = malloc(sizeof(double) * D), *mubar = malloc(sizeof(double) * D);
  int rc = ORA_OK;
  if (!xbar || !Sbar || !Al || !al || !Kd || !Ko || !b || !mubar) { rc = ORA_ENOMEM; goto done; }
  ora_init_mean(pb, xbar);
  ora_init_mean(pb, mu);
  for (int i = 0; i <= N; ++i) memcpy(Sbar + i * nn, pb->K0, sizeof(double) * nn);
  ora_problem hot = *pb;
  hot.temperature = op->temperature_high;
  for (int j = 0; j < op->slr_iters; ++j) {
    double logdet;
    const ora_problem *cur = hot_phase(op, j * op->iters) ? &hot : pb;
    if ((rc = ora_slr(pb, op, xbar, Sbar, Al, al))) goto done;
    if ((rc = ora_prior(cur, Al, al, Kd, Ko, b, NULL, NULL, NULL))) goto done;
    if ((rc = ora_prior_mean(cur, Kd, Ko, b, mubar))) goto done;
    if (j == 0) {
      memcpy(Ld, Kd, sizeof(double) * (N + 1) * nn);
      memcpy(Lo, Ko, sizeof(double) * N * nn);
    }
    if ((rc = ora_marginals(n, N, Ld, Lo, Sd, So, &logdet))) goto done;
    for (int k = 0; k < op->iters; ++k) {
      if (hot_phase(op, j * op->iters + k) && cur == pb) {   /* switch inside this linearisation */
        cur = &hot;
        if ((rc = ora_prior(cur, Al, al, Kd, Ko, b, NULL, NULL, NULL))) goto done;
        if ((rc = ora_prior_mean(cur, Kd, Ko, b, mubar))) goto done;
      }
      if ((rc = ora_step(cur, op, j * op->iters + k, Kd, Ko, b, mubar, mu, Ld, Lo, Sd, So, &logdet,
                         logs ? logs + (size_t)j * op->iters + k : NULL)))
        goto done;
    }
    double s = 0.0;
    for (int e = 0; e < D; ++e) s += (mu[e] - xbar[e]) * (mu[e] - xbar[e]);
    if (slr_norms) slr_norms[j] = sqrt(s);
    memcpy(xbar, mu, sizeof(double) * D);
    memcpy(Sbar, Sd, sizeof(double) * (N + 1) * nn);
  }
done:
  free(xbar); free(Sbar); free(Al); free(al); free(Kd); free(Ko); free(b); free(mubar);
  return rc;
}
