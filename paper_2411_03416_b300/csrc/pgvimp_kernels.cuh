// pgvimp_kernels.cu -- the P-GVIMP hot path on sm_103a, one plan per thread.
//
// Rows of the path and where they live:
//   prior build (Alg. 1, lines 1-2)         prior_build<n>       / k_prior
//   marginals by GBP on the chain (Sec. 5.1) marginals<n>        / k_init, k_marginals
//   factor expectations (Sec. 4.1-4.3)      quad_factor<n, QT>   / k_quad, k_iterate
//   gradient assembly (Sec. 4.2)            quad_factor<n, QT>
//   Thm 1 update + step search (App. C)     trial<n>, search<n>  / k_trial, k_iterate
//   SLR linearisation (Sec. 6.2, Alg. 2)    slr_step<n, QT>      / k_slr
//
// GBP on a chain is the exact two-pass message schedule; here the forward
// messages are carried as Schur-complement pivots C_i (the precision of x_i
// given x_{<i} marginalised), and the backward messages as the covariance
// recursion Sigma_i = C_i^-1 + W_i^T Sigma_{i+1} W_i, Sigma_{i+1,i} =
// -Sigma_{i+1} W_i with W_i = Lambda_{i+1,i} C_i^-1.  Both carry only PSD sums
// in the backward direction, which keeps FP64 accuracy at N ~ 1000.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "pgvimp_device.cuh"

namespace pgv {

template <int n>
__host__ __device__ constexpr int scr_stride() { return 3 * n * n + n; }

PGV_DEV double ln_2pie() { return 2.8378770664093454836; }  // 1 + ln(2 pi)

// ------------------------------------------------------------ prior (a0)

// Van Loan: expm([[-A, W],[0, A^T]] dt) = [[., G12],[0, G22]], Phi = G22^T,
// Q = Phi G12; u = top-right column of expm([[A, a],[0, 0]] dt).
template <int n>
PGV_BIG bool van_loan(const double* A, const double* a, const double* Wn, double dt, double* Phi, double* Q,
                      double* u) {
  constexpr int D = 2 * n;
  double H[D * D], E[D * D];
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) H[r * D + c] = 0.0;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      H[r * D + c] = -A[r * n + c] * dt;
      H[r * D + n + c] = Wn[r * n + c] * dt;
      H[(n + r) * D + n + c] = A[c * n + r] * dt;
    }
  if (!expm_pade6<D>(D, H, E)) return false;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Phi[r * n + c] = E[(n + c) * D + n + r];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s = fma(Phi[r * n + k], E[k * D + n + c], s);
      Q[r * n + c] = s;
    }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < r; ++c) {
      double s = 0.5 * (Q[r * n + c] + Q[c * n + r]);
      Q[r * n + c] = s;
      Q[c * n + r] = s;
    }
  constexpr int D1 = n + 1;
  double Ha[D1 * D1], Ea[D1 * D1];
  for (int r = 0; r < D1; ++r)
    for (int c = 0; c < D1; ++c) Ha[r * D1 + c] = 0.0;
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) Ha[r * D1 + c] = A[r * n + c] * dt;
    Ha[r * D1 + n] = a[r] * dt;
  }
  if (!expm_pade6<D1>(D1, Ha, Ea)) return false;
  for (int r = 0; r < n; ++r) u[r] = Ea[r * D1 + n];
  return true;
}

// Block-tridiagonal solve M x = r (M symmetric positive definite, diagonal
// blocks Md, lower blocks Mo) by the same forward elimination / back
// substitution as the trial sweep; scratch from P.scr.
template <int n>
PGV_BIG bool bt_solve(const PlanDesc& P, const double* Md, const double* Mo, const double* r, double* x) {
  constexpr int nn = n * n, SS = scr_stride<n>();
  const int N = P.N;
  double S[nn], C[nn], Ci[nn], E[nn], Wm[nn], y[n], yp[n], z[n];
  LogDetAcc ld;
  ld.init();
  bool ok = true;
  for (int e = 0; e < nn; ++e) S[e] = 0.0;
  for (int a = 0; a < n; ++a) yp[a] = 0.0;
  for (int e = 0; e < nn; ++e) Wm[e] = 0.0;
  for (int i = 0; i <= N; ++i) {
    ld_blk<n>(Md + (size_t)i * nn, C);
    for (int e = 0; e < nn; ++e) C[e] -= S[e];
    ok = chol_inverse<n>(C, Ci, ld) && ok;
    for (int a = 0; a < n; ++a) {
      double s = r[(size_t)i * n + a];
      for (int c = 0; c < n; ++c) s = fma(-Wm[a * n + c], yp[c], s);
      y[a] = s;
    }
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(Ci[a * n + c], y[c], s);
      z[a] = s;
    }
    double* sp = P.scr + (size_t)i * SS;
    st_vec<n>(sp + 3 * nn, z);
    if (i < N) {
      ld_blk<n>(Mo + (size_t)i * nn, E);
      mul_nn<n>(E, Ci, Wm);
      mul_nt_sym<n>(Wm, E, S);
      st_blk<n>(sp + nn, Wm);
    }
    for (int a = 0; a < n; ++a) yp[a] = y[a];
  }
  double xn[n];
  ld_vec<n>(P.scr + (size_t)N * SS + 3 * nn, xn);
  st_vec<n>(x + (size_t)N * n, xn);
  for (int i = N - 1; i >= 0; --i) {
    const double* sp = P.scr + (size_t)i * SS;
    ld_blk<n>(sp + nn, Wm);
    ld_vec<n>(sp + 3 * nn, z);
    double xi[n];
    for (int a = 0; a < n; ++a) {
      double s = z[a];
      for (int c = 0; c < n; ++c) s = fma(-Wm[c * n + a], xn[c], s);
      xi[a] = s;
    }
    st_vec<n>(x + (size_t)i * n, xi);
    for (int a = 0; a < n; ++a) xn[a] = xi[a];
  }
  return ok;
}

// Prior precision K^-1 (block tridiagonal), information vector b = K^-1 mu_bar
// and mu_bar itself, for the LTI / LTV system given by (A, a) or, when Altv
// is non-null, by the SLR linearisation (Altv, altv).
template <int n>
PGV_BIG bool prior_build(const PlanDesc& P, bool use_ltv) {
  constexpr int nn = n * n;
  const int N = P.N, m = P.m;
  double Wn[nn], Phi[nn], Q[nn], Qi[nn], u[n], A[nn], av[n];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < m; ++k)
        for (int l = 0; l < m; ++l) s += P.B[r * m + k] * P.Qc[k * m + l] * P.B[c * m + l];
      Wn[r * n + c] = s;
    }
  const bool lti = !use_ltv && !P.A_per_step && !P.a_per_step;
  double carry_d[nn], carry_b[n], PtQi[nn], T1[nn];
  LogDetAcc dummy;
  dummy.init();
  bool ok = true;
  // start factor
  {
    double K0i[nn];
    double K0[nn];
    for (int e = 0; e < nn; ++e) K0[e] = P.K0[e];
    ok = chol_inverse<n>(K0, K0i, dummy) && ok;
    for (int e = 0; e < nn; ++e) carry_d[e] = K0i[e];
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(K0i[a * n + c], P.mu0[c], s);
      carry_b[a] = s;
    }
  }
  const double it = P.inv_temp;
  for (int i = 0; i < N; ++i) {
    if (i == 0 || !lti) {
      const double* Ai = use_ltv ? P.Altv + (size_t)i * nn : (P.A_per_step ? P.A + (size_t)i * nn : P.A);
      for (int e = 0; e < nn; ++e) A[e] = Ai[e];
      for (int a = 0; a < n; ++a)
        av[a] = use_ltv ? P.altv[(size_t)i * n + a] : (P.a ? (P.a_per_step ? P.a[(size_t)i * n + a] : P.a[a]) : 0.0);
      ok = van_loan<n>(A, av, Wn, P.dt, Phi, Q, u) && ok;
      ok = chol_inverse<n>(Q, Qi, dummy) && ok;
      // PtQi = Phi^T Q^-1
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double s = 0.0;
          for (int k = 0; k < n; ++k) s = fma(Phi[k * n + r], Qi[k * n + c], s);
          PtQi[r * n + c] = s;
        }
    }
    // K^-1_ii = carry + Phi^T Q^-1 Phi ; b_i = carry_b - Phi^T Q^-1 u
    mul_nn<n>(PtQi, Phi, T1);
    double blk[nn], bv[n];
    for (int e = 0; e < nn; ++e) blk[e] = (carry_d[e] + T1[e]) * it;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < r; ++c) {
        double s = 0.5 * (blk[r * n + c] + blk[c * n + r]);
        blk[r * n + c] = s;
        blk[c * n + r] = s;
      }
    st_blk<n>(P.Kd + (size_t)i * nn, blk);
    for (int a = 0; a < n; ++a) {
      double s = carry_b[a];
      for (int c = 0; c < n; ++c) s = fma(-PtQi[a * n + c], u[c], s);
      bv[a] = s * it;
    }
    st_vec<n>(P.b + (size_t)i * n, bv);
    // K^-1_{i+1,i} = -Q^-1 Phi
    mul_nn<n>(Qi, Phi, T1);
    for (int e = 0; e < nn; ++e) blk[e] = -T1[e] * it;
    st_blk<n>(P.Ko + (size_t)i * nn, blk);
    for (int e = 0; e < nn; ++e) carry_d[e] = Qi[e];
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(Qi[a * n + c], u[c], s);
      carry_b[a] = s;
    }
  }
  {
    double KN[nn], KNi[nn], blk[nn], bv[n];
    for (int e = 0; e < nn; ++e) KN[e] = P.KN[e];
    ok = chol_inverse<n>(KN, KNi, dummy) && ok;
    for (int e = 0; e < nn; ++e) blk[e] = (carry_d[e] + KNi[e]) * it;
    st_blk<n>(P.Kd + (size_t)N * nn, blk);
    for (int a = 0; a < n; ++a) {
      double s = carry_b[a];
      for (int c = 0; c < n; ++c) s = fma(KNi[a * n + c], P.muN[c], s);
      bv[a] = s * it;
    }
    st_vec<n>(P.b + (size_t)N * n, bv);
  }
  if (ok) ok = bt_solve<n>(P, P.Kd, P.Ko, P.b, P.mubar);
  return ok;
}

// ------------------------------------------------------------ marginals (a1)

// Marginal blocks of the block-tridiagonal precision (Ld, Lo) into set s, the
// log det, and the prior cost 1/2[tr(K^-1 Sigma) + (mu-mubar)^T K^-1 (mu-mubar)]
// of the iterate (mu[s], Sigma).
template <int n>
PGV_BIG bool marginals(const PlanDesc& P, const double* Ld, const double* Lo, int s, double& logdet,
                       double& prior_cost) {
  constexpr int nn = n * n, SS = scr_stride<n>();
  const int N = P.N;
  double S[nn], C[nn], Ci[nn], E[nn], W[nn];
  LogDetAcc ld;
  ld.init();
  bool ok = true;
  for (int e = 0; e < nn; ++e) S[e] = 0.0;
  for (int i = 0; i <= N; ++i) {
    ld_blk<n>(Ld + (size_t)i * nn, C);
    for (int e = 0; e < nn; ++e) C[e] -= S[e];
    ok = chol_inverse<n>(C, Ci, ld) && ok;
    double* sp = P.scr + (size_t)i * SS;
    st_blk<n>(sp, Ci);
    if (i < N) {
      ld_blk<n>(Lo + (size_t)i * nn, E);
      mul_nn<n>(E, Ci, W);
      mul_nt_sym<n>(W, E, S);
      st_blk<n>(sp + nn, W);
    }
  }
  logdet = ld.log_value();
  if (!ok) return false;
  double Sn[nn], T[nn], Si[nn], K[nn], dn[n], di[n];
  const double* mu = P.mu[s];
  ld_blk<n>(P.scr + (size_t)N * SS, Sn);
  st_blk<n>(P.Sd[s] + (size_t)N * nn, Sn);
  double tr = 0.0, qd = 0.0;
  ld_blk<n>(P.Kd + (size_t)N * nn, K);
  for (int a = 0; a < n; ++a) dn[a] = mu[(size_t)N * n + a] - P.mubar[(size_t)N * n + a];
  for (int e = 0; e < nn; ++e) tr = fma(K[e], Sn[e], tr);
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) qd = fma(dn[a] * K[a * n + c], dn[c], qd);
  for (int i = N - 1; i >= 0; --i) {
    const double* sp = P.scr + (size_t)i * SS;
    ld_blk<n>(sp, Ci);
    ld_blk<n>(sp + nn, W);
    mul_nn<n>(Sn, W, T);
    add_tn_sym<n>(Ci, W, T, Si);
    for (int e = 0; e < nn; ++e) T[e] = -T[e];
    st_blk<n>(P.So[s] + (size_t)i * nn, T);
    st_blk<n>(P.Sd[s] + (size_t)i * nn, Si);
    ld_blk<n>(P.Kd + (size_t)i * nn, K);
    ld_blk<n>(P.Ko + (size_t)i * nn, E);
    for (int a = 0; a < n; ++a) di[a] = mu[(size_t)i * n + a] - P.mubar[(size_t)i * n + a];
    for (int e = 0; e < nn; ++e) tr = fma(K[e], Si[e], fma(2.0 * E[e], T[e], tr));
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        qd = fma(di[a] * K[a * n + c], di[c], qd);
        qd = fma(2.0 * dn[a] * E[a * n + c], di[c], qd);
      }
    for (int e = 0; e < nn; ++e) Sn[e] = Si[e];
    for (int a = 0; a < n; ++a) dn[a] = di[a];
  }
  prior_cost = 0.5 * (tr + qd);
  return true;
}

// Prior cost of the iterate in set s (used after a relinearisation changes K^-1).
template <int n>
PGV_BIG double prior_cost_of(const PlanDesc& P, int s) {
  constexpr int nn = n * n;
  const int N = P.N;
  double tr = 0.0, qd = 0.0, K[nn], E[nn], Sb[nn], Ob[nn], di[n], dn[n];
  for (int i = N; i >= 0; --i) {
    ld_blk<n>(P.Kd + (size_t)i * nn, K);
    ld_blk<n>(P.Sd[s] + (size_t)i * nn, Sb);
    for (int a = 0; a < n; ++a) di[a] = P.mu[s][(size_t)i * n + a] - P.mubar[(size_t)i * n + a];
    for (int e = 0; e < nn; ++e) tr = fma(K[e], Sb[e], tr);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) qd = fma(di[a] * K[a * n + c], di[c], qd);
    if (i < N) {
      ld_blk<n>(P.Ko + (size_t)i * nn, E);
      ld_blk<n>(P.So[s] + (size_t)i * nn, Ob);
      for (int e = 0; e < nn; ++e) tr = fma(2.0 * E[e], Ob[e], tr);
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) qd = fma(2.0 * dn[a] * E[a * n + c], di[c], qd);
    }
    for (int a = 0; a < n; ++a) dn[a] = di[a];
  }
  return 0.5 * (tr + qd);
}

// ------------------------------------------------------- quadrature (a2-a4)

// Collision cost at a state whose cost coordinates are mu_a + dx_a.  The grid
// coordinate of the mean is pre-split into integer base + fraction (gb, gf).
template <typename QT>
PGV_DEV QT point_psi(const PlanDesc& P, const int* gb, const QT* gf, const QT* dx, const QT* mu_a) {
  const QT ic = (QT)P.inv_cell;
  if (P.cost_kind == PGVIMP_COST_POINT2D) {
    QT s = sdf2<QT>(P.sdf, P.nx, P.ny, gb[0], gf[0] + dx[0] * ic, gb[1], gf[1] + dx[1] * ic);
    return hinge_psi<QT>(P, (QT)P.eps - s);
  }
  if (P.cost_kind == PGVIMP_COST_POINT3D) {
    QT s = sdf3<QT>(P.sdf, P.nx, P.ny, P.nz, gb[0], gf[0] + dx[0] * ic, gb[1], gf[1] + dx[1] * ic, gb[2],
                    gf[2] + dx[2] * ic);
    return hinge_psi<QT>(P, (QT)P.eps - s);
  }
  // arm: joint angles
  QT q[kMaxDof];
  for (int a = 0; a < P.arm_dof; ++a) q[a] = mu_a[a] + dx[a];
  return arm_cost<QT>(P, q);
}

// E[psi_i] and the gradients g_i = Sigma^-1 E[(x-mu) psi],
// G_i = -1/2 Sigma^-1 E[psi] + 1/2 Sigma^-1 E[(x-mu)(x-mu)^T psi] Sigma^-1
// (Sec. 4.1 moment form) for one factor.  With x = mu + L xi and L lower
// triangular, the cost (a function of the leading dc coordinates) depends on
// xi_0..xi_{dc-1} only, so the quadrature runs over the dc-dimensional rule
// in xi-space: g = L^-T E[xi psi], G = 1/2 L^-T (E[xi xi^T psi] - E[psi] I) L^-1,
// where the trailing moments are known in closed form (tensor GH: xi_b
// independent of psi; degree 3: +-sqrt(3) e_b points evaluate psi(mu)).
template <int n, typename QT>
PGV_DEV bool quad_factor(const PlanDesc& P, int i, const double* mu_i, const double* S_ii, double* g,
                         double* G, double& M0_out) {
  constexpr int nn = n * n;
  for (int a = 0; a < n; ++a) g[a] = 0.0;
  for (int e = 0; e < nn; ++e) G[e] = 0.0;
  M0_out = 0.0;
  if (P.cost_kind == PGVIMP_COST_NONE || (P.factor_set == 1 && (i == 0 || i == P.N))) return true;
  const int dc = P.dc;
  const bool deg3 = (P.rule == PGVIMP_RULE_DEG3);
  const int dL = deg3 ? n : dc;
  double L[nn], Li[nn];
  if (!chol_lead<n, double>(S_ii, dL, L, Li)) return false;
  QT Lq[nn], mua[kMaxN];
  for (int e = 0; e < nn; ++e) Lq[e] = (QT)L[e];
  for (int a = 0; a < dc; ++a) mua[a] = (QT)mu_i[a];
  int gb[3] = {0, 0, 0};
  QT gf[3] = {0, 0, 0};
  if (P.cost_kind != PGVIMP_COST_ARM) {
    for (int a = 0; a < dc; ++a) {
      double u = (mu_i[a] - P.sdf_origin[a]) * P.inv_cell;
      double fl = floor(u);
      gb[a] = (int)fl;
      gf[a] = (QT)(u - fl);
    }
  }
  QT M0 = 0, M1[kMaxN], M2[kMaxN * kMaxN];
  for (int a = 0; a < dc; ++a) M1[a] = 0;
  for (int e = 0; e < dc * dc; ++e) M2[e] = 0;
  QT dx[kMaxN], psi_c = 0;
  if (!deg3) {
    const int p = P.gh_p;
    int Pn = 1;
    for (int a = 0; a < dc; ++a) Pn *= p;
    for (int l = 0; l < Pn; ++l) {
      QT xi[kMaxN];
      QT w = 1;
      int rem = l;
      for (int a = dc - 1; a >= 0; --a) {
        int d = rem % p;
        rem /= p;
        xi[a] = (QT)P.gh_x[p * kMaxGH + d];
        w *= (QT)P.gh_w[p * kMaxGH + d];
      }
      for (int a = 0; a < dc; ++a) {
        QT s = 0;
        for (int c = 0; c <= a; ++c) s += Lq[a * n + c] * xi[c];
        dx[a] = s;
      }
      QT wp = w * point_psi<QT>(P, gb, gf, dx, mua);
      M0 += wp;
      for (int a = 0; a < dc; ++a) {
        QT t = wp * xi[a];
        M1[a] += t;
        for (int c = 0; c <= a; ++c) M2[a * dc + c] += t * xi[c];
      }
    }
  } else {
    for (int a = 0; a < dc; ++a) dx[a] = 0;
    psi_c = point_psi<QT>(P, gb, gf, dx, mua);
    M0 = (QT)(1.0 - dc / 3.0) * psi_c;
    const QT r3 = (QT)1.7320508075688772935, w6 = (QT)(1.0 / 6.0);
    for (int j = 0; j < dc; ++j) {
      for (int a = 0; a < dc; ++a) dx[a] = r3 * Lq[a * n + j];
      QT pp = point_psi<QT>(P, gb, gf, dx, mua);
      for (int a = 0; a < dc; ++a) dx[a] = -r3 * Lq[a * n + j];
      QT pm = point_psi<QT>(P, gb, gf, dx, mua);
      M0 += w6 * (pp + pm);
      M1[j] = w6 * r3 * (pp - pm);
      M2[j * dc + j] = (QT)0.5 * (pp + pm);
    }
  }
  // gradient assembly in FP64: D = blockdiag(M2 - M0 I, (psi_c - M0) I [deg3 only])
  // (the cost is divided by the temperature T-hat)
  const double it = P.inv_temp;
  double D[nn];
  for (int e = 0; e < nn; ++e) D[e] = 0.0;
  const double m0 = (double)M0 * it;
  for (int a = 0; a < dc; ++a)
    for (int c = 0; c <= a; ++c) {
      double v = (double)M2[a * dc + c] * it - (a == c ? m0 : 0.0);
      D[a * n + c] = v;
      D[c * n + a] = v;
    }
  if (deg3)
    for (int b = dc; b < n; ++b) D[b * n + b] = (double)psi_c * it - m0;
  // g = Li^T m1
  for (int r = 0; r < dL; ++r) {
    double s = 0.0;
    for (int a = r; a < dc; ++a) s = fma(Li[a * n + r], (double)M1[a] * it, s);
    g[r] = s;
  }
  // G = 1/2 Li^T D Li  (Li lower triangular, dL x dL)
  double T[nn];
  for (int a = 0; a < dL; ++a)
    for (int c = 0; c < dL; ++c) {
      double s = 0.0;
      for (int b = c; b < dL; ++b) s = fma(D[a * n + b], Li[b * n + c], s);
      T[a * n + c] = s;
    }
  for (int r = 0; r < dL; ++r)
    for (int c = 0; c <= r; ++c) {
      double s = 0.0;
      for (int a = r; a < dL; ++a) s = fma(Li[a * n + r], T[a * n + c], s);
      G[r * n + c] = 0.5 * s;
      G[c * n + r] = 0.5 * s;
    }
  M0_out = m0;
  return true;
}

template <int n, typename QT>
PGV_BIG bool quad_all(const PlanDesc& P, int s, double& coll) {
  constexpr int nn = n * n;
  const int N = P.N;
  double mu_i[n], S_ii[nn], g[n], G[nn], m0;
  coll = 0.0;
  bool ok = true;
  for (int i = 0; i <= N; ++i) {
    ld_vec<n>(P.mu[s] + (size_t)i * n, mu_i);
    ld_blk<n>(P.Sd[s] + (size_t)i * nn, S_ii);
    ok = quad_factor<n, QT>(P, i, mu_i, S_ii, g, G, m0) && ok;
    st_vec<n>(P.g + (size_t)i * n, g);
    st_blk<n>(P.G + (size_t)i * nn, G);
    coll += m0;
  }
  return ok;
}

// ------------------------------------------------------------ trial (a5)

struct TrialOut {
  double kl, logdet, prior_cost, delta, trace;
  bool pd;
};

// Thm 1 at step beta, scaled by (beta+1):
//   A~ = beta (2G + K^-1) + Lambda_k          = (beta+1) Lambda'
//   M  = beta K^-1 + Lambda_k                 (mean system times beta)
//   M delta = beta (-g + b - K^-1 mu_k),      mu' = mu_k + delta
// One forward sweep eliminates A~ and M together (they share the
// off-diagonal blocks); one backward sweep produces Sigma~ = A~^-1 (selected
// blocks), delta, and the KL pieces
//   KL = 1/2 [beta tr((Lambda_k - 2G - K^-1) Sigma~) + delta^T Lambda_k delta
//             + log det Lambda' - log det Lambda_k],
// using tr(Lambda_k Sigma') - D = tr((Lambda_k - Lambda') Sigma').
// Results go to buffer set `out`: mu', Sigma' = (beta+1) Sigma~.
template <int n>
PGV_BIG TrialOut trial(const PlanDesc& P, double beta, int cur, int out, double logdet_k) {
  constexpr int nn = n * n, SS = scr_stride<n>();
  const int N = P.N;
  const double* mu = P.mu[cur];
  TrialOut R;
  R.kl = INFINITY;
  R.pd = false;
  R.logdet = 0.0;
  R.prior_cost = 0.0;
  R.delta = 0.0;
  R.trace = 0.0;
  double SA[nn], SM[nn], WMp[nn], yp[n];
  for (int e = 0; e < nn; ++e) { SA[e] = 0.0; SM[e] = 0.0; WMp[e] = 0.0; }
  for (int a = 0; a < n; ++a) yp[a] = 0.0;
  LogDetAcc ldA, ldM;
  ldA.init();
  ldM.init();
  bool okA = true, okM = true;
  double mprev[n], mi[n], mnext[n];
  for (int a = 0; a < n; ++a) mprev[a] = 0.0;
  ld_vec<n>(mu, mi);
  for (int i = 0; i <= N; ++i) {
    double Kd[nn], Lb[nn], Gb[nn], CA[nn], CM[nn], CiA[nn], CiM[nn];
    ld_blk<n>(P.Kd + (size_t)i * nn, Kd);
    ld_blk<n>(P.Ld + (size_t)i * nn, Lb);
    ld_blk<n>(P.G + (size_t)i * nn, Gb);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int e = 0; e < nn; ++e) {
      double kb = beta * Kd[e];
      CM[e] = kb + Lb[e] - SM[e];
      CA[e] = fma(2.0 * beta, Gb[e], kb) + Lb[e] - SA[e];
    }
    okA = chol_inverse<n>(CA, CiA, ldA) && okA;
    okM = chol_inverse<n>(CM, CiM, ldM) && okM;
    // r_i = beta (-g_i + b_i - (K^-1 mu)_i)
    double Kmu[n];
    if (i < N) ld_vec<n>(mu + (size_t)(i + 1) * n, mnext);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int c = 0; c < n; ++c) s = fma(Kd[a * n + c], mi[c], s);
      Kmu[a] = s;
    }
    if (i > 0) {
      double Eo[nn];
      ld_blk<n>(P.Ko + (size_t)(i - 1) * nn, Eo);
#pragma unroll (n <= 8 ? 32 : 1)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
        for (int c = 0; c < n; ++c) Kmu[a] = fma(Eo[a * n + c], mprev[c], Kmu[a]);
    }
    double En[nn], Kon[nn];
    if (i < N) {
      ld_blk<n>(P.Ko + (size_t)i * nn, Kon);
      ld_blk<n>(P.Lo + (size_t)i * nn, En);
#pragma unroll (n <= 8 ? 32 : 1)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
        for (int c = 0; c < n; ++c) Kmu[a] = fma(Kon[c * n + a], mnext[c], Kmu[a]);
    }
    double y[n], z[n];
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      double r = beta * (-P.g[(size_t)i * n + a] + P.b[(size_t)i * n + a] - Kmu[a]);
#pragma unroll (n <= 8 ? 32 : 1)
      for (int c = 0; c < n; ++c) r = fma(-WMp[a * n + c], yp[c], r);
      y[a] = r;
    }
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int c = 0; c < n; ++c) s = fma(CiM[a * n + c], y[c], s);
      z[a] = s;
    }
    double* sp = P.scr + (size_t)i * SS;
    st_blk<n>(sp, CiA);
    st_vec<n>(sp + 3 * nn, z);
    if (i < N) {
      double WA[nn];
#pragma unroll (n <= 8 ? 32 : 1)
      for (int e = 0; e < nn; ++e) En[e] = fma(beta, Kon[e], En[e]);
      mul_nn<n>(En, CiA, WA);
      mul_nn<n>(En, CiM, WMp);
      mul_nt_sym<n>(WA, En, SA);
      mul_nt_sym<n>(WMp, En, SM);
      st_blk<n>(sp + nn, WA);
      st_blk<n>(sp + 2 * nn, WMp);
    }
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      yp[a] = y[a];
      mprev[a] = mi[a];
      mi[a] = mnext[a];
    }
  }
  if (!okA || !okM) return R;
  R.pd = true;
  const double D = (double)n * (N + 1);
  const double bp1 = beta + 1.0;
  R.logdet = ldA.log_value() - D * log(bp1);
  // backward sweep
  double Sn[nn], xn[n];
  double trc = 0.0, dl = 0.0, ktr = 0.0, kq = 0.0, dpn[n];
  {
    const double* sp = P.scr + (size_t)N * SS;
    ld_blk<n>(sp, Sn);
    ld_vec<n>(sp + 3 * nn, xn);
    double Kd[nn], Lb[nn], Gb[nn];
    ld_blk<n>(P.Kd + (size_t)N * nn, Kd);
    ld_blk<n>(P.Ld + (size_t)N * nn, Lb);
    ld_blk<n>(P.G + (size_t)N * nn, Gb);
    for (int e = 0; e < nn; ++e) {
      trc = fma(Lb[e] - 2.0 * Gb[e] - Kd[e], Sn[e], trc);
      ktr = fma(Kd[e], Sn[e], ktr);
    }
    double mo[n];
    for (int a = 0; a < n; ++a) {
      mo[a] = mu[(size_t)N * n + a] + xn[a];
      dpn[a] = mo[a] - P.mubar[(size_t)N * n + a];
    }
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        dl = fma(xn[a] * Lb[a * n + c], xn[c], dl);
        kq = fma(dpn[a] * Kd[a * n + c], dpn[c], kq);
      }
    st_blk_scaled<n>(P.Sd[out] + (size_t)N * nn, Sn, bp1);
    st_vec<n>(P.mu[out] + (size_t)N * n, mo);
  }
  for (int i = N - 1; i >= 0; --i) {
    const double* sp = P.scr + (size_t)i * SS;
    double CiA[nn], WA[nn], WM[nn], z[n], T[nn], Si[nn], xi[n];
    ld_blk<n>(sp, CiA);
    ld_blk<n>(sp + nn, WA);
    ld_blk<n>(sp + 2 * nn, WM);
    ld_vec<n>(sp + 3 * nn, z);
    mul_nn<n>(Sn, WA, T);
    add_tn_sym<n>(CiA, WA, T, Si);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      double s = z[a];
#pragma unroll (n <= 8 ? 32 : 1)
      for (int c = 0; c < n; ++c) s = fma(-WM[c * n + a], xn[c], s);
      xi[a] = s;
    }
    double Kd[nn], Lb[nn], Gb[nn], Ko[nn], Lo[nn];
    ld_blk<n>(P.Kd + (size_t)i * nn, Kd);
    ld_blk<n>(P.Ld + (size_t)i * nn, Lb);
    ld_blk<n>(P.G + (size_t)i * nn, Gb);
    ld_blk<n>(P.Ko + (size_t)i * nn, Ko);
    ld_blk<n>(P.Lo + (size_t)i * nn, Lo);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int e = 0; e < nn; ++e) {
      // Sigma~_{i+1,i} = -T
      trc = fma(Lb[e] - 2.0 * Gb[e] - Kd[e], Si[e], trc);
      trc = fma(-2.0 * (Lo[e] - Ko[e]), T[e], trc);
      ktr = fma(Kd[e], Si[e], fma(-2.0 * Ko[e], T[e], ktr));
    }
    double mo[n], dpi[n];
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      mo[a] = mu[(size_t)i * n + a] + xi[a];
      dpi[a] = mo[a] - P.mubar[(size_t)i * n + a];
    }
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
      for (int c = 0; c < n; ++c) {
        dl = fma(xi[a] * Lb[a * n + c], xi[c], dl);
        dl = fma(2.0 * xn[a] * Lo[a * n + c], xi[c], dl);
        kq = fma(dpi[a] * Kd[a * n + c], dpi[c], kq);
        kq = fma(2.0 * dpn[a] * Ko[a * n + c], dpi[c], kq);
      }
    st_blk_scaled<n>(P.Sd[out] + (size_t)i * nn, Si, bp1);
    st_blk_scaled<n>(P.So[out] + (size_t)i * nn, T, -bp1);
    st_vec<n>(P.mu[out] + (size_t)i * n, mo);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int e = 0; e < nn; ++e) Sn[e] = Si[e];
#pragma unroll (n <= 8 ? 32 : 1)
    for (int a = 0; a < n; ++a) {
      xn[a] = xi[a];
      dpn[a] = dpi[a];
    }
  }
  R.trace = beta * trc;
  R.delta = dl;
  R.kl = 0.5 * (R.trace + dl + R.logdet - logdet_k);
  R.prior_cost = 0.5 * (bp1 * ktr + kq);
  return R;
}

// Lambda_{k+1} = A~(beta) / (beta+1), written over (Ld, Lo).
template <int n>
PGV_BIG void accept_precision(const PlanDesc& P, double beta) {
  constexpr int nn = n * n;
  const int N = P.N;
  const double inv = 1.0 / (beta + 1.0);
  for (int i = 0; i <= N; ++i) {
    double Kd[nn], Lb[nn], Gb[nn];
    ld_blk<n>(P.Kd + (size_t)i * nn, Kd);
    ld_blk<n>(P.Ld + (size_t)i * nn, Lb);
    ld_blk<n>(P.G + (size_t)i * nn, Gb);
    for (int e = 0; e < nn; ++e) Lb[e] = (fma(beta, fma(2.0, Gb[e], Kd[e]), Lb[e])) * inv;
    st_blk<n>(P.Ld + (size_t)i * nn, Lb);
    if (i < N) {
      double Ko[nn], Lo[nn];
      ld_blk<n>(P.Ko + (size_t)i * nn, Ko);
      ld_blk<n>(P.Lo + (size_t)i * nn, Lo);
      for (int e = 0; e < nn; ++e) Lo[e] = fma(beta, Ko[e], Lo[e]) * inv;
      st_blk<n>(P.Lo + (size_t)i * nn, Lo);
    }
  }
}

// One proximal iteration (Alg. 1 loop body) for the plan: quadrature and
// gradients at the current iterate, the largest feasible step by bisection
// (App. C: beta_max first, then max_bisect halvings of [0, beta_max]; feasible
// = Lambda' positive definite and KL <= eps), and the update.
template <int n, typename QT>
PGV_BIG void iterate_once(const PlanDesc& P) {
  double* sc = P.scal;
  const int cur = (int)sc[S_CUR];
  const int oa = (cur + 1) % 3, ob = (cur + 2) % 3;
  double coll;
  if (!quad_all<n, QT>(P, cur, coll)) {
    sc[S_STATUS] = 3.0;
    return;
  }
  const double logdet_k = sc[S_LOGDET];
  const double eps = P.kl_eps;
  const bool has_eps = isfinite(eps) && eps > 0.0;
  double margin = INFINITY;
  int trials = 0, best = -1;
  TrialOut bestR;
  double best_beta = 0.0;
  bestR.kl = 0.0;
  bestR.logdet = logdet_k;
  bestR.prior_cost = sc[S_PRIOR];
  // beta_max first; if infeasible, max_bisect halvings of [0, beta_max]
  double beta = P.beta_max, lo = 0.0, hi = P.beta_max;
  int into = oa, halvings = 0;
  bool searching = false;
  for (;;) {
    TrialOut R = trial<n>(P, beta, cur, into, logdet_k);
    ++trials;
    if (R.pd && has_eps) margin = fmin(margin, fabs(R.kl - eps) / eps);
    const bool feas = R.pd && (R.kl <= eps);
    if (feas) {
      best = into;
      best_beta = beta;
      bestR = R;
    }
    if (!searching) {
      if (feas) break;
      searching = true;
    } else {
      if (feas) lo = beta;
      else hi = beta;
      ++halvings;
    }
    if (halvings >= P.max_bisect) break;
    beta = 0.5 * (lo + hi);
    into = (best == oa) ? ob : oa;
  }
  const int k = (int)sc[S_K];
  if (k < P.log_cap) {
    pgvimp_step_info li;
    li.beta = best_beta;
    li.kl = (best >= 0) ? bestR.kl : 0.0;
    li.kl_margin = margin;
    li.prior_cost = sc[S_PRIOR];
    li.collision_cost = coll;
    li.entropy = 0.5 * ((double)P.n * (P.N + 1) * ln_2pie() - logdet_k);
    li.trials = trials;
    li.iter = k;
    P.log[k] = li;
  }
  if (best >= 0) {
    accept_precision<n>(P, best_beta);
    sc[S_CUR] = (double)best;
    sc[S_LOGDET] = bestR.logdet;
    sc[S_PRIOR] = bestR.prior_cost;
  }
  sc[S_COLL] = coll;
  sc[S_K] = (double)(k + 1);
  sc[S_KIN] = sc[S_KIN] + 1.0;
}

// Initial iterate (mu_0 straight line in q with constant qdot; Lambda_0 = K^-1
// or init_scale * I) and its marginals.
template <int n>
PGV_BIG void init_plan(const PlanDesc& P) {
  constexpr int nn = n * n;
  double* sc = P.scal;
  const int N = P.N, nq = P.nq;
  for (int i = 0; i <= N; ++i) {
    double s = (double)i / N;
    for (int a = 0; a < nq; ++a) {
      double d = P.muN[a] - P.mu0[a];
      P.mu[0][(size_t)i * n + a] = P.mu0[a] + s * d;
      P.mu[0][(size_t)i * n + nq + a] = d / P.T;
    }
  }
  for (int i = 0; i <= N; ++i) {
    double blk[nn];
    if (P.init_kind == 1) {
      for (int e = 0; e < nn; ++e) blk[e] = 0.0;
      for (int a = 0; a < n; ++a) blk[a * n + a] = P.init_scale;
    } else {
      ld_blk<n>(P.Kd + (size_t)i * nn, blk);
    }
    st_blk<n>(P.Ld + (size_t)i * nn, blk);
    if (i < N) {
      if (P.init_kind == 1)
        for (int e = 0; e < nn; ++e) blk[e] = 0.0;
      else
        ld_blk<n>(P.Ko + (size_t)i * nn, blk);
      st_blk<n>(P.Lo + (size_t)i * nn, blk);
    }
  }
  double ld, pc;
  if (!marginals<n>(P, P.Ld, P.Lo, 0, ld, pc)) {
    sc[S_STATUS] = 2.0;
    return;
  }
  sc[S_CUR] = 0.0;
  sc[S_LOGDET] = ld;
  sc[S_PRIOR] = pc;
  sc[S_K] = 0.0;
  sc[S_KIN] = 0.0;
  sc[S_INIT] = 1.0;
}

// ------------------------------------------------------------ SLR (a6)

// Planar quadrotor prior drift f_0(x) (eq. planar_quad with u = 0).
template <typename QT>
PGV_DEV void quad_drift(QT g, const QT* x, QT* f) {
  QT s, c;
  if (sizeof(QT) == 4) { float sf, cf; sincosf((float)x[2], &sf, &cf); s = sf; c = cf; }
  else { double sd, cd; sincos((double)x[2], &sd, &cd); s = (QT)sd; c = (QT)cd; }
  const QT vx = x[3], vz = x[4], w = x[5];
  f[0] = vx * c - vz * s;
  f[1] = vx * s + vz * c;
  f[2] = w;
  f[3] = vz * w - g * s;
  f[4] = -vx * w - g * c;
  f[5] = 0;
}

// A_i = P_yx P_xx^-1, a_i = E f - A_i E x (Sec. 6.2) by quadrature over
// N(xbar_i, Sbar_i).  With x = xbar + L xi and a symmetric rule exact to
// degree 2: E x = xbar, P_xx = Sbar, P_yx = E[f xi^T] L^T, so A_i = E[f xi^T] L^-1.
template <int n, typename QT>
PGV_DEV bool slr_step(const PlanDesc& P, const double* xbar, const double* Sbar, double* Aout, double* aout) {
  constexpr int nn = n * n;
  double L[nn], Li[nn];
  if (!chol_lead<n, double>(Sbar, n, L, Li)) return false;
  QT Lq[nn], xb[n];
  for (int e = 0; e < nn; ++e) Lq[e] = (QT)L[e];
  for (int a = 0; a < n; ++a) xb[a] = (QT)xbar[a];
  QT Ef[n], F1[nn];
  for (int a = 0; a < n; ++a) Ef[a] = 0;
  for (int e = 0; e < nn; ++e) F1[e] = 0;
  const QT g = (QT)P.dyn_params[3];
  auto accum = [&](const QT* xi, QT w) {
    QT x[n], f[n];
    for (int a = 0; a < n; ++a) {
      QT s = xb[a];
      for (int c = 0; c <= a; ++c) s += Lq[a * n + c] * xi[c];
      x[a] = s;
    }
    quad_drift<QT>(g, x, f);
    for (int a = 0; a < n; ++a) {
      QT wf = w * f[a];
      Ef[a] += wf;
      for (int c = 0; c < n; ++c) F1[a * n + c] += wf * xi[c];
    }
  };
  if (P.rule == PGVIMP_RULE_DEG3) {
    QT xi[n];
    for (int a = 0; a < n; ++a) xi[a] = 0;
    accum(xi, (QT)(1.0 - n / 3.0));
    const QT r3 = (QT)1.7320508075688772935;
    for (int j = 0; j < n; ++j) {
      xi[j] = r3;
      accum(xi, (QT)(1.0 / 6.0));
      xi[j] = -r3;
      accum(xi, (QT)(1.0 / 6.0));
      xi[j] = 0;
    }
  } else {
    const int p = P.gh_p;
    int Pn = 1;
    for (int a = 0; a < n; ++a) Pn *= p;
    for (int l = 0; l < Pn; ++l) {
      QT xi[n];
      QT w = 1;
      int rem = l;
      for (int a = n - 1; a >= 0; --a) {
        int d = rem % p;
        rem /= p;
        xi[a] = (QT)P.gh_x[p * kMaxGH + d];
        w *= (QT)P.gh_w[p * kMaxGH + d];
      }
      accum(xi, w);
    }
  }
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = c; k < n; ++k) s = fma((double)F1[a * n + k], Li[k * n + c], s);
      Aout[a * n + c] = s;
    }
  for (int a = 0; a < n; ++a) {
    double s = (double)Ef[a];
    for (int c = 0; c < n; ++c) s = fma(-Aout[a * n + c], xbar[c], s);
    aout[a] = s;
  }
  return true;
}

template <int n, typename QT>
PGV_BIG bool slr_all(const PlanDesc& P, bool first) {
  constexpr int nn = n * n;
  const int N = P.N, nq = P.nq;
  double xb[n], Sb[nn];
  bool ok = true;
  for (int i = 0; i < N; ++i) {
    if (first) {
      double s = (double)i / N;
      for (int a = 0; a < nq; ++a) {
        double d = P.muN[a] - P.mu0[a];
        xb[a] = P.mu0[a] + s * d;
        xb[nq + a] = d / P.T;
      }
      for (int e = 0; e < nn; ++e) Sb[e] = P.K0[e];
    } else {
      const int cur = (int)P.scal[S_CUR];
      ld_vec<n>(P.mu[cur] + (size_t)i * n, xb);
      ld_blk<n>(P.Sd[cur] + (size_t)i * nn, Sb);
    }
    st_vec<n>(P.xbar + (size_t)i * n, xb);
    ok = slr_step<n, QT>(P, xb, Sb, P.Altv + (size_t)i * nn, P.altv + (size_t)i * n) && ok;
  }
  if (first) {
    double s = 1.0;
    for (int a = 0; a < nq; ++a) {
      double d = P.muN[a] - P.mu0[a];
      xb[a] = P.mu0[a] + s * d;
      xb[nq + a] = d / P.T;
    }
    st_vec<n>(P.xbar + (size_t)N * n, xb);
  } else {
    const int cur = (int)P.scal[S_CUR];
    ld_vec<n>(P.mu[cur] + (size_t)N * n, xb);
    st_vec<n>(P.xbar + (size_t)N * n, xb);
  }
  return ok;
}

// ------------------------------------------------------------ kernels

#define PLAN_OR_RETURN                                     \
  const int t = blockIdx.x * blockDim.x + threadIdx.x;     \
  if (t >= count) return;                                  \
  const PlanDesc& P = descs[t];

// Prior build; `mode` 0: linear system (A, a); 1: the SLR linearisation.
template <int n>
__global__ void k_prior(const PlanDesc* __restrict__ descs, int count, int mode) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  if (!prior_build<n>(P, mode == 1)) P.scal[S_STATUS] = 1.0;
}

template <int n>
__global__ void k_init(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  init_plan<n>(P);
}

// After a relinearisation: the prior cost of the current iterate under the
// new prior, and a fresh inner-iteration counter.
template <int n>
__global__ void k_relinearised(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  P.scal[S_PRIOR] = prior_cost_of<n>(P, (int)P.scal[S_CUR]);
  P.scal[S_KIN] = 0.0;
}

template <int n, typename QT>
__global__ void __launch_bounds__(64) k_iterate(const PlanDesc* __restrict__ descs, int count, int iters) {
  PLAN_OR_RETURN
  for (int it = 0; it < iters; ++it) {
    if (P.scal[S_STATUS] != 0.0 || P.scal[S_INIT] == 0.0) return;
    if ((int)P.scal[S_KIN] >= P.iters) return;
    iterate_once<n, QT>(P);
  }
}

// SLR linearisation.  mode 1: the straight-line nominal with K0 (first
// outer iteration); 0: the current iterate, closing the previous outer
// iteration (its norm); 2: the current iterate without bookkeeping.
template <int n, typename QT>
__global__ void k_slr(const PlanDesc* __restrict__ descs, int count, int mode) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  const int first = (mode == 1);
  if (mode == 0) {
    // ||xbar^{j+1} - xbar^j||: the finished linearisation's result vs its nominal
    const int cur = (int)P.scal[S_CUR];
    const int j = (int)P.scal[S_J];
    double s = 0.0;
    for (size_t e = 0; e < (size_t)(P.N + 1) * n; ++e) {
      double d = P.mu[cur][e] - P.xbar[e];
      s = fma(d, d, s);
    }
    if (j < P.slr_iters) P.slr_norms[j] = sqrt(s);
    P.scal[S_J] = (double)(j + 1);
  }
  if (!slr_all<n, QT>(P, first != 0)) P.scal[S_STATUS] = 4.0;
}

// Final SLR norm after the last linearisation's iterations.
template <int n>
__global__ void k_slr_finish(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  const int cur = (int)P.scal[S_CUR];
  const int j = (int)P.scal[S_J];
  double s = 0.0;
  for (size_t e = 0; e < (size_t)(P.N + 1) * n; ++e) {
    double d = P.mu[cur][e] - P.xbar[e];
    s = fma(d, d, s);
  }
  if (j < P.slr_iters) P.slr_norms[j] = sqrt(s);
  P.scal[S_J] = (double)(j + 1);
}

// Moves the current iterate into buffer set 0 (the one results are read from).
template <int n>
__global__ void k_finalize(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  const int cur = (int)P.scal[S_CUR];
  if (cur == 0) return;
  const size_t N = P.N;
  for (size_t e = 0; e < (N + 1) * n; ++e) P.mu[0][e] = P.mu[cur][e];
  for (size_t e = 0; e < (N + 1) * n * n; ++e) P.Sd[0][e] = P.Sd[cur][e];
  for (size_t e = 0; e < N * n * n; ++e) P.So[0][e] = P.So[cur][e];
  P.scal[S_CUR] = 0.0;
}

// Single-row phases (for per-row checks through the C ABI).
template <int n>
__global__ void k_marginals(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  double ld, pc;
  const int cur = (int)P.scal[S_CUR];
  bool ok = marginals<n>(P, P.Ld, P.Lo, cur, ld, pc);
  P.scal[S_LOGDET] = ld;
  P.scal[S_PRIOR] = pc;
  if (!ok) P.scal[S_STATUS] = 2.0;
}

template <int n, typename QT>
__global__ void k_quad(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  double coll;
  bool ok = quad_all<n, QT>(P, (int)P.scal[S_CUR], coll);
  P.scal[S_COLL] = coll;
  if (!ok) P.scal[S_STATUS] = 3.0;
}

template <int n>
__global__ void k_trial(const PlanDesc* __restrict__ descs, int count, double beta) {
  PLAN_OR_RETURN
  const int cur = (int)P.scal[S_CUR];
  TrialOut R = trial<n>(P, beta, cur, (cur + 2) % 3, P.scal[S_LOGDET]);
  P.scal[S_T_LOGDET] = R.logdet;
  P.scal[S_T_KL] = R.kl;
  P.scal[S_T_PD] = R.pd ? 1.0 : 0.0;
  P.scal[S_T_PRIOR] = R.prior_cost;
  P.scal[S_T_DELTA] = R.delta;
  P.scal[S_T_TRACE] = R.trace;
}

// ------------------------------------------------------------ launchers

static inline int blocks_for(int count, int tpb) { return (count + tpb - 1) / tpb; }

// Launch groups; each is instantiated in its own translation unit so that the
// (fully inlined) kernels of one state dimension compile in parallel.
//   iter<n, QT>: the fused proximal iterations (Alg. 1 loop);
//   aux<n>:      prior build, initial iterate, SLR, bookkeeping kernels;
//   rows<n>:     the single-row kernels (marginals, quadrature, one trial).
enum { PH_PRIOR = 100, PH_INIT = 101, PH_ITER = 102, PH_SLR = 103, PH_RELIN = 104, PH_SLR_FIN = 105,
       PH_FINALIZE = 106 };

template <int n, typename QT>
cudaError_t launch_iter(const Launch& L, int iters) {
  const int tpb = 32;
  k_iterate<n, QT><<<blocks_for(L.count, tpb), tpb, 0, L.stream>>>(L.descs, L.count, iters);
  return cudaGetLastError();
}

template <int n>
cudaError_t launch_aux(const Launch& L, int phase, int arg_i, int mixed) {
  const int tpb = 32;
  dim3 g(blocks_for(L.count, tpb)), b(tpb);
  switch (phase) {
    case PH_PRIOR: k_prior<n><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i); break;
    case PH_INIT: k_init<n><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_SLR:
      if (mixed) k_slr<n, float><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i);
      else k_slr<n, double><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i);
      break;
    case PH_RELIN: k_relinearised<n><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_SLR_FIN: k_slr_finish<n><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_FINALIZE: k_finalize<n><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int n>
cudaError_t launch_rows(const Launch& L, int phase, double arg_d, int mixed) {
  const int tpb = 32;
  dim3 g(blocks_for(L.count, tpb)), b(tpb);
  switch (phase) {
    case PGVIMP_PHASE_MARGINALS: k_marginals<n><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PGVIMP_PHASE_QUAD:
      if (mixed) k_quad<n, float><<<g, b, 0, L.stream>>>(L.descs, L.count);
      else k_quad<n, double><<<g, b, 0, L.stream>>>(L.descs, L.count);
      break;
    case PGVIMP_PHASE_TRIAL: k_trial<n><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_d); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pgv
