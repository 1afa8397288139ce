// pgvimp_kernels.cuh -- the P-GVIMP hot path on sm_103a, one plan per thread.
//
// Rows of the path and where they live:
//   prior build (Alg. 1, its set-up)         prior_build<n, R>        / k_prior
//   marginals on the chain (Sec. 5.1)        marginals<n, R>          / k_init, k_marginals
//   factor expectations (Sec. 4.1-4.3)       quad_factor<n, QT, R>    / k_quad, k_iterate
//   gradient assembly (Sec. 4.2)             quad_factor<n, QT, R>
//   Thm 1 update + step search (App. C)      trial<n, R>, iterate_once / k_trial, k_iterate
//   SLR linearisation (Sec. 6.2, Alg. 2)     slr_step<n, QT>          / k_slr
//
// QT is the quadrature arithmetic (float in the mixed forms, double in the
// plain FP64 form); R the arithmetic and storage of the block recursions
// (double, or the double-float df64).
//
// Gaussian belief propagation on a chain is the exact two-pass schedule; here
// the forward messages are carried as Schur-complement pivots C_i (the
// precision of x_i after the states before it are marginalised out) and the
// backward messages as the covariance recursion
//   Sigma_i = C_i^-1 + W_i^T Sigma_{i+1} W_i,  Sigma_{i+1,i} = -Sigma_{i+1} W_i,
// with W_i = Lambda_{i+1,i} C_i^-1.  The backward direction adds only PSD
// terms, which keeps the marginals accurate at N ~ 1000.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "pgvimp_device.cuh"

namespace pgv {

// Per-state scratch of a sweep (elements of R): packed C_A^-1, W_A, W_M, z.
template <int n>
struct Scr {
  static constexpr int np = n * (n + 1) / 2;
  static constexpr int npe = np + (np & 1);
  static constexpr int oCi = 0, oWA = npe, oWM = npe + n * n, oZ = npe + 2 * n * n;
  static constexpr int stride = npe + 2 * n * n + n;
};

PGV_DEV double ln_2pie() { return 2.8378770664093454836; }  // 1 + ln(2 pi)

template <typename R>
PGV_DEV R* rp(double* p) { return reinterpret_cast<R*>(p); }
template <typename R>
PGV_DEV const R* rp(const double* p) { return reinterpret_cast<const R*>(p); }

template <int n, typename R>
PGV_DEV void st_blk_from_double(R* p, const double* X) {
  R Y[n * n];
  for (int e = 0; e < n * n; ++e) Y[e] = r_from<R>(X[e]);
  st_blk<n, R>(p, Y);
}

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

// Inverse of an SPD n x n block (full, FP64) through the packed Cholesky.
template <int n>
PGV_DEV bool spd_inverse_full(const double* A, double* Ai) {
  constexpr int np = n * (n + 1) / 2;
  double P[np], Pi[np];
  for (int a = 0; a < n; ++a)
    for (int c = 0; c <= a; ++c) P[pk(a, c)] = A[a * n + c];
  LogDetAcc<double> ld;
  ld.init();
  bool ok = true;
  chol_inverse<n, double>(P, Pi, ld, ok);
  for (int a = 0; a < n; ++a)
    for (int c = 0; c < n; ++c) Ai[a * n + c] = Pi[pk(a, c)];
  return ok;
}

// Block-tridiagonal SPD solve M x = r (diagonal blocks Md, lower blocks Mo)
// by forward elimination and back substitution; scratch from P.scr.
template <int n, typename R>
PGV_BIG bool bt_solve(const PlanDesc& P, const R* Md, const R* Mo, const R* r, R* x) {
  constexpr int nn = n * n, np = Scr<n>::np, SS = Scr<n>::stride;
  const int N = P.N;
  R* scr = rp<R>(P.scr);
  R S[np], v[n];
  const R zero = r_fromf<R>(0.0f);
  for (int e = 0; e < np; ++e) S[e] = zero;
  for (int a = 0; a < n; ++a) v[a] = zero;
  LogDetAcc<R> ld;
  ld.init();
  bool ok = true;
  for (int i = 0; i <= N; ++i) {
    R C[np], Ci[np], y[n], z[n];
    ld_sym<n, R>(Md + (size_t)i * nn, C);
    for (int e = 0; e < np; ++e) C[e] = C[e] - S[e];
    chol_inverse<n, R>(C, Ci, ld, ok);
    for (int a = 0; a < n; ++a) y[a] = r[(size_t)i * n + a] - v[a];
    for (int a = 0; a < n; ++a) {
      R s = Ci[pk(a, 0)] * y[0];
      for (int c = 1; c < n; ++c) s = r_fma(Ci[pk(a, c)], y[c], s);
      z[a] = s;
    }
    R* sp = scr + (size_t)i * SS;
    st_vec<n, R>(sp + Scr<n>::oZ, z);
    if (i < N) {
      R E[nn], W[nn];
      ld_blk<n, R>(Mo + (size_t)i * nn, E);
      mul_full_sym<n, R>(E, Ci, W);
      mul_nt_packed<n, R>(W, E, S);
      for (int a = 0; a < n; ++a) {
        R s = W[a * n] * y[0];
        for (int c = 1; c < n; ++c) s = r_fma(W[a * n + c], y[c], s);
        v[a] = s;
      }
      st_blk<n, R>(sp + Scr<n>::oWA, W);
    }
  }
  R xn[n];
  ld_vec<n, R>(scr + (size_t)N * SS + Scr<n>::oZ, xn);
  st_vec<n, R>(x + (size_t)N * n, xn);
  for (int i = N - 1; i >= 0; --i) {
    const R* sp = scr + (size_t)i * SS;
    R W[nn], z[n], xi[n];
    ld_blk<n, R>(sp + Scr<n>::oWA, W);
    ld_vec<n, R>(sp + Scr<n>::oZ, z);
    for (int a = 0; a < n; ++a) {
      R s = z[a];
      for (int c = 0; c < n; ++c) s = r_fma(-W[c * n + a], xn[c], s);
      xi[a] = s;
    }
    st_vec<n, R>(x + (size_t)i * n, xi);
    for (int a = 0; a < n; ++a) xn[a] = xi[a];
  }
  return ok;
}

// Inverse temperature at the plan's current global iteration: the problem's
// T-hat, or the high temperature from iteration switch_iter on.
PGV_DEV double cur_inv_temp(const PlanDesc& P) {
  return (P.inv_temp_high > 0.0 && P.scal[S_K] >= (double)P.switch_iter) ? P.inv_temp_high : P.inv_temp;
}

// Prior precision K^-1 (block tridiagonal), information vector b = K^-1 mu_bar
// and mu_bar, for the LTI / LTV system given by (A, a) or, with `use_ltv`, by
// the SLR linearisation (Altv, altv).  FP64 throughout; stored as R.
template <int n, typename R>
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
  bool ok = true;
  R* Kd = rp<R>(P.Kd);
  R* Ko = rp<R>(P.Ko);
  R* b = rp<R>(P.b);
  {
    double K0i[nn];
    ok = spd_inverse_full<n>(P.K0, K0i) && ok;
    for (int e = 0; e < nn; ++e) carry_d[e] = K0i[e];
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(K0i[a * n + c], P.mu0[c], s);
      carry_b[a] = s;
    }
  }
  const double it = cur_inv_temp(P);
  P.scal[S_THIGH] = (P.inv_temp_high > 0.0 && it == P.inv_temp_high) ? 1.0 : 0.0;
  for (int i = 0; i < N; ++i) {
    if (i == 0 || !lti) {
      const double* Ai = use_ltv ? P.Altv + (size_t)i * nn : (P.A_per_step ? P.A + (size_t)i * nn : P.A);
      for (int e = 0; e < nn; ++e) A[e] = Ai[e];
      for (int a = 0; a < n; ++a)
        av[a] = use_ltv ? P.altv[(size_t)i * n + a] : (P.a ? (P.a_per_step ? P.a[(size_t)i * n + a] : P.a[a]) : 0.0);
      ok = van_loan<n>(A, av, Wn, P.dt, Phi, Q, u) && ok;
      ok = spd_inverse_full<n>(Q, Qi) && ok;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double s = 0.0;
          for (int k = 0; k < n; ++k) s = fma(Phi[k * n + r], Qi[k * n + c], s);
          PtQi[r * n + c] = s;
        }
    }
    // K^-1_ii = carry + Phi^T Q^-1 Phi ; b_i = carry_b - Phi^T Q^-1 u
    double blk[nn], bv[n];
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(PtQi[r * n + k], Phi[k * n + c], s);
        T1[r * n + c] = s;
      }
    for (int e = 0; e < nn; ++e) blk[e] = (carry_d[e] + T1[e]) * it;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < r; ++c) {
        double s = 0.5 * (blk[r * n + c] + blk[c * n + r]);
        blk[r * n + c] = s;
        blk[c * n + r] = s;
      }
    st_blk_from_double<n, R>(Kd + (size_t)i * nn, blk);
    for (int a = 0; a < n; ++a) {
      double s = carry_b[a];
      for (int c = 0; c < n; ++c) s = fma(-PtQi[a * n + c], u[c], s);
      bv[a] = s * it;
    }
    for (int a = 0; a < n; ++a) b[(size_t)i * n + a] = r_from<R>(bv[a]);
    // K^-1_{i+1,i} = -Q^-1 Phi
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s = fma(Qi[r * n + k], Phi[k * n + c], s);
        blk[r * n + c] = -s * it;
      }
    st_blk_from_double<n, R>(Ko + (size_t)i * nn, blk);
    for (int e = 0; e < nn; ++e) carry_d[e] = Qi[e];
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s = fma(Qi[a * n + c], u[c], s);
      carry_b[a] = s;
    }
  }
  {
    double KNi[nn], blk[nn];
    ok = spd_inverse_full<n>(P.KN, KNi) && ok;
    for (int e = 0; e < nn; ++e) blk[e] = (carry_d[e] + KNi[e]) * it;
    st_blk_from_double<n, R>(Kd + (size_t)N * nn, blk);
    for (int a = 0; a < n; ++a) {
      double s = carry_b[a];
      for (int c = 0; c < n; ++c) s = fma(KNi[a * n + c], P.muN[c], s);
      b[(size_t)N * n + a] = r_from<R>(s * it);
    }
  }
  if (ok) ok = bt_solve<n, R>(P, Kd, Ko, b, rp<R>(P.mubar));
  return ok;
}

// ------------------------------------------------------------ marginals (a1)

// Marginal blocks of the precision (Ld, Lo) into buffer set s, log det, and
// the prior cost 1/2 [tr(K^-1 Sigma) + (mu - mubar)^T K^-1 (mu - mubar)] of
// the iterate (mu[s], Sigma).
template <int n, typename R>
PGV_BIG bool marginals(const PlanDesc& P, int s, double& logdet, double& prior_cost) {
  constexpr int nn = n * n, np = Scr<n>::np, SS = Scr<n>::stride;
  const int N = P.N;
  const R* Ld = rp<R>(P.Ld);
  const R* Lo = rp<R>(P.Lo);
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* mubar = rp<R>(P.mubar);
  const R* mu = rp<R>(P.mu[s]);
  R* Sd = rp<R>(P.Sd[s]);
  R* So = rp<R>(P.So[s]);
  R* scr = rp<R>(P.scr);
  R S[np];
  const R zero = r_fromf<R>(0.0f);
  for (int e = 0; e < np; ++e) S[e] = zero;
  LogDetAcc<R> ld;
  ld.init();
  bool ok = true;
  for (int i = 0; i <= N; ++i) {
    R C[np], Ci[np];
    ld_sym<n, R>(Ld + (size_t)i * nn, C);
    for (int e = 0; e < np; ++e) C[e] = C[e] - S[e];
    chol_inverse<n, R>(C, Ci, ld, ok);
    R* sp = scr + (size_t)i * SS;
    st_packed<n, R>(sp + Scr<n>::oCi, Ci);
    if (i < N) {
      R E[nn], W[nn];
      ld_blk<n, R>(Lo + (size_t)i * nn, E);
      mul_full_sym<n, R>(E, Ci, W);
      mul_nt_packed<n, R>(W, E, S);
      st_blk<n, R>(sp + Scr<n>::oWA, W);
    }
  }
  logdet = ld.log_value();
  if (!ok) return false;
  R Sn[np], dn[n];
  ld_packed<n, R>(scr + (size_t)N * SS + Scr<n>::oCi, Sn);
  st_sym<n, R>(Sd + (size_t)N * nn, Sn);
  R tr = zero, qd = zero;
  {
    R K[nn];
    ld_blk<n, R>(Kd + (size_t)N * nn, K);
    for (int a = 0; a < n; ++a) dn[a] = mu[(size_t)N * n + a] - mubar[(size_t)N * n + a];
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        tr = r_fma(K[a * n + c], Sn[pk(a, c)], tr);
        qd = r_fma(dn[a] * K[a * n + c], dn[c], qd);
      }
  }
  for (int i = N - 1; i >= 0; --i) {
    const R* sp = scr + (size_t)i * SS;
    R Ci[np], W[nn], T[nn], Si[np], di[n];
    ld_packed<n, R>(sp + Scr<n>::oCi, Ci);
    ld_blk<n, R>(sp + Scr<n>::oWA, W);
    mul_sym_full<n, R>(Sn, W, T);           // Sigma_{i+1} W_i = -Sigma_{i+1,i}
    add_tn_packed<n, R>(Ci, W, T, Si);
    for (int e = 0; e < nn; ++e) T[e] = -T[e];
    st_blk<n, R>(So + (size_t)i * nn, T);
    st_sym<n, R>(Sd + (size_t)i * nn, Si);
    R K[nn], E[nn];
    ld_blk<n, R>(Kd + (size_t)i * nn, K);
    ld_blk<n, R>(Ko + (size_t)i * nn, E);
    for (int a = 0; a < n; ++a) di[a] = mu[(size_t)i * n + a] - mubar[(size_t)i * n + a];
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        tr = r_fma(K[a * n + c], Si[pk(a, c)], tr);
        tr = r_fma(E[a * n + c] + E[a * n + c], T[a * n + c], tr);
        qd = r_fma(di[a] * K[a * n + c], di[c], qd);
        qd = r_fma((dn[a] + dn[a]) * E[a * n + c], di[c], qd);
      }
    for (int e = 0; e < np; ++e) Sn[e] = Si[e];
    for (int a = 0; a < n; ++a) dn[a] = di[a];
  }
  prior_cost = 0.5 * r_to(tr + qd);
  return true;
}

// Prior cost of the iterate in set s (after a relinearisation changes K^-1).
template <int n, typename R>
PGV_BIG double prior_cost_of(const PlanDesc& P, int s) {
  constexpr int nn = n * n;
  const int N = P.N;
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* mu = rp<R>(P.mu[s]);
  const R* mubar = rp<R>(P.mubar);
  const R* Sd = rp<R>(P.Sd[s]);
  const R* So = rp<R>(P.So[s]);
  R tr = r_fromf<R>(0.0f), qd = r_fromf<R>(0.0f), di[n], dn[n];
  for (int i = N; i >= 0; --i) {
    R K[nn], Sb[nn];
    ld_blk<n, R>(Kd + (size_t)i * nn, K);
    ld_blk<n, R>(Sd + (size_t)i * nn, Sb);
    for (int a = 0; a < n; ++a) di[a] = mu[(size_t)i * n + a] - mubar[(size_t)i * n + a];
    for (int e = 0; e < nn; ++e) tr = r_fma(K[e], Sb[e], tr);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) qd = r_fma(di[a] * K[a * n + c], di[c], qd);
    if (i < N) {
      R E[nn], Ob[nn];
      ld_blk<n, R>(Ko + (size_t)i * nn, E);
      ld_blk<n, R>(So + (size_t)i * nn, Ob);
      for (int e = 0; e < nn; ++e) tr = r_fma(E[e] + E[e], Ob[e], tr);
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) qd = r_fma((dn[a] + dn[a]) * E[a * n + c], di[c], qd);
    }
    for (int a = 0; a < n; ++a) dn[a] = di[a];
  }
  return 0.5 * r_to(tr + qd);
}

// ------------------------------------------------------- quadrature (a2-a4)

// The point robots' cost constants in the quadrature's arithmetic, converted
// once per factor rather than at every sigma point (on B300 each FP64 -> FP32
// conversion occupies the narrow FP64 pipe).
template <typename QT>
struct QuadConsts {
  QT inv_cell, eps, w;   // 1/cell, hinge margin, weight of h^2
};
template <typename QT>
PGV_DEV QuadConsts<QT> quad_consts(const PlanDesc& P) {
  QuadConsts<QT> k;
  k.inv_cell = (QT)P.inv_cell;
  k.eps = (QT)P.eps;
  k.w = (P.psi_form == 1) ? (QT)(1.0 / (P.sigma_obs * P.sigma_obs)) : (QT)P.sigma_obs;
  return k;
}

// Collision cost at a state whose cost coordinates are mu_a + dx_a.  The grid
// coordinate of the mean is pre-split into integer base + fraction (gb, gf).
template <typename QT>
PGV_DEV QT point_psi(const PlanDesc& P, const QuadConsts<QT>& k, const int* gb, const QT* gf, const QT* dx,
                     const QT* mu_a) {
  const QT ic = k.inv_cell;
  if (P.cost_kind == PGVIMP_COST_POINT2D || P.cost_kind == PGVIMP_COST_POINT3D) {
    QT s = (P.cost_kind == PGVIMP_COST_POINT2D)
               ? sdf2<QT>(P.sdf, P.nx, P.ny, gb[0], gf[0] + dx[0] * ic, gb[1], gf[1] + dx[1] * ic)
               : sdf3<QT>(P.sdf, P.nx, P.ny, P.nz, gb[0], gf[0] + dx[0] * ic, gb[1], gf[1] + dx[1] * ic, gb[2],
                          gf[2] + dx[2] * ic);
    QT h = k.eps - s;
    h = h > (QT)0 ? h : (QT)0;
    return k.w * h * h;
  }
  QT q[kMaxDof];
  for (int a = 0; a < P.arm_dof; ++a) q[a] = mu_a[a] + dx[a];
  return arm_cost<QT>(P, q);
}

// A recursion value in the quadrature's arithmetic (double-float to FP32 by
// one FP32 add, no FP64 operation).
template <typename QT>
PGV_DEV QT r_toq(double v) { return (QT)v; }
template <typename QT>
PGV_DEV QT r_toq(df64 v);
template <>
PGV_DEV float r_toq<float>(df64 v) { return __fadd_rn(v.hi, v.lo); }
template <>
PGV_DEV double r_toq<double>(df64 v) { return r_to(v); }

// Grid coordinate (mu - origin)/cell split into an exact integer part and a
// fraction, evaluated in the recursion's arithmetic.
template <typename QT>
PGV_DEV void grid_split(double mu, double origin, double inv_cell, int& base, QT& frac) {
  double u = (mu - origin) * inv_cell;
  double fl = floor(u);
  base = (int)fl;
  frac = (QT)(u - fl);
}
template <typename QT>
PGV_DEV void grid_split(df64 mu, double origin, double inv_cell, int& base, QT& frac) {
  df64 u = (mu - r_from<df64>(origin)) * r_from<df64>(inv_cell);
  float fl = floorf(u.hi);
  base = (int)fl;
  frac = (QT)((u.hi - fl) + u.lo);
}

// A moment (quadrature arithmetic) times the inverse temperature, in the
// recursion's arithmetic: FP64 as a double product; double-float as the exact
// float value times the double-float inverse temperature (no FP64 operation).
PGV_DEV double scale_moment(float m, double it, double) { return (double)m * it; }
PGV_DEV double scale_moment(double m, double it, double) { return m * it; }
PGV_DEV df64 scale_moment(float m, double, df64 itr) { return df_make(m, 0.0f) * itr; }

// E[psi_i] and the gradients g_i = Sigma^-1 E[(x-mu) psi],
// G_i = -1/2 Sigma^-1 E[psi] + 1/2 Sigma^-1 E[(x-mu)(x-mu)^T psi] Sigma^-1
// (Sec. 4.1 moment form) for one factor.  With x = mu + L xi and L lower
// triangular, the cost (a function of the leading dc coordinates) depends on
// xi_0..xi_{dc-1} only, so the quadrature runs over the dc-dimensional rule in
// xi-space: g = L^-T E[xi psi], G = 1/2 L^-T (E[xi xi^T psi] - E[psi] I) L^-1,
// the trailing moments being known in closed form (tensor GH: xi_b is
// independent of psi; degree 3: the +-sqrt(3) e_b points evaluate psi(mu);
// Smolyak of level k: the n-dimensional grid restricted to the dc cost
// coordinates is the dc-dimensional grid of the same level, and a trailing
// xi_b^2 psi integrates to the level k-1 value).
template <int n, typename QT, typename R>
PGV_DEV bool quad_factor(const PlanDesc& P, int i, const R* mu_i, const R* S_ii, R* g, R* G, double& M0_out) {
  constexpr int nn = n * n;
  const R zero = r_fromf<R>(0.0f);
  for (int a = 0; a < n; ++a) g[a] = zero;
  for (int e = 0; e < nn; ++e) G[e] = zero;
  M0_out = 0.0;
  if (P.cost_kind == PGVIMP_COST_NONE || (P.factor_set == 1 && (i == 0 || i == P.N))) return true;
  const int dc = P.dc;
  const bool deg3 = (P.rule == PGVIMP_RULE_DEG3);
  const bool sparse = (P.rule == PGVIMP_RULE_SMOLYAK);
  const int dL = (deg3 || sparse) ? n : dc;
  R L[nn], Li[nn];
  if (!chol_lead<n, R>(S_ii, dL, L, Li)) return false;
  QT Lq[nn], mua[kMaxN];
  for (int e = 0; e < nn; ++e) Lq[e] = r_toq<QT>(L[e]);
  for (int a = 0; a < dc; ++a) mua[a] = r_toq<QT>(mu_i[a]);
  const QuadConsts<QT> kq = quad_consts<QT>(P);
  int gb[3] = {0, 0, 0};
  QT gf[3] = {0, 0, 0};
  if (P.cost_kind != PGVIMP_COST_ARM)
    for (int a = 0; a < dc; ++a) grid_split<QT>(mu_i[a], P.sdf_origin[a], P.inv_cell, gb[a], gf[a]);
  QT M0 = 0, M1[kMaxN], M2[kMaxN * kMaxN];
  for (int a = 0; a < dc; ++a) M1[a] = 0;
  for (int e = 0; e < dc * dc; ++e) M2[e] = 0;
  QT dx[kMaxN], psi_c = 0;
  if (sparse) {
    const int cols = dc + 2;
    for (int l = 0; l < P.sg_rows; ++l) {
      const double* row = P.sg + (size_t)l * cols;
      QT xi[kMaxN];
      for (int a = 0; a < dc; ++a) xi[a] = (QT)row[a];
      for (int a = 0; a < dc; ++a) {
        QT s = 0;
        for (int c = 0; c <= a; ++c) s += Lq[a * n + c] * xi[c];
        dx[a] = s;
      }
      const QT ps = point_psi<QT>(P, kq, gb, gf, dx, mua);
      const QT wp = (QT)row[dc] * ps;
      psi_c += (QT)row[dc + 1] * ps;          // level k-1: the trailing second moments
      M0 += wp;
      for (int a = 0; a < dc; ++a) {
        QT t = wp * xi[a];
        M1[a] += t;
        for (int c = 0; c <= a; ++c) M2[a * dc + c] += t * xi[c];
      }
    }
  } else if (!deg3) {
    const int p = P.gh_p;
    int Pn = 1;
    for (int a = 0; a < dc; ++a) Pn *= p;
    QT xq[kMaxGH], wq[kMaxGH];   // the 1-D rule, converted once
    for (int d = 0; d < p; ++d) {
      xq[d] = (QT)P.gh_x[p * kMaxGH + d];
      wq[d] = (QT)P.gh_w[p * kMaxGH + d];
    }
    for (int l = 0; l < Pn; ++l) {
      QT xi[kMaxN];
      QT w = 1;
      int rem = l;
      for (int a = dc - 1; a >= 0; --a) {
        int d = rem % p;
        rem /= p;
        xi[a] = xq[d];
        w *= wq[d];
      }
      for (int a = 0; a < dc; ++a) {
        QT s = 0;
        for (int c = 0; c <= a; ++c) s += Lq[a * n + c] * xi[c];
        dx[a] = s;
      }
      QT wp = w * point_psi<QT>(P, kq, gb, gf, dx, mua);
      M0 += wp;
      for (int a = 0; a < dc; ++a) {
        QT t = wp * xi[a];
        M1[a] += t;
        for (int c = 0; c <= a; ++c) M2[a * dc + c] += t * xi[c];
      }
    }
  } else {
    for (int a = 0; a < dc; ++a) dx[a] = 0;
    psi_c = point_psi<QT>(P, kq, gb, gf, dx, mua);
    M0 = (QT)(1.0 - dc / 3.0) * psi_c;
    const QT r3 = (QT)1.7320508075688772935, w6 = (QT)(1.0 / 6.0);
    for (int j = 0; j < dc; ++j) {
      for (int a = 0; a < dc; ++a) dx[a] = r3 * Lq[a * n + j];
      QT pp = point_psi<QT>(P, kq, gb, gf, dx, mua);
      for (int a = 0; a < dc; ++a) dx[a] = -r3 * Lq[a * n + j];
      QT pm = point_psi<QT>(P, kq, gb, gf, dx, mua);
      M0 += w6 * (pp + pm);
      M1[j] = w6 * r3 * (pp - pm);
      M2[j * dc + j] = (QT)0.5 * (pp + pm);
    }
  }
  // gradient assembly: D = blockdiag(M2 - M0 I, (psi_c - M0) I [degree 3 only]);
  // the cost is divided by the temperature T-hat
  const double it = cur_inv_temp(P);
  const R itr = r_from<R>(it);
  R D[nn];
  for (int e = 0; e < nn; ++e) D[e] = zero;
  const double m0 = (double)M0 * it;
  const R m0r = scale_moment(M0, it, itr);
  for (int a = 0; a < dc; ++a)
    for (int c = 0; c <= a; ++c) {
      R v = scale_moment(M2[a * dc + c], it, itr);
      if (a == c) v = v - m0r;
      D[a * n + c] = v;
      D[c * n + a] = v;
    }
  if (deg3 || sparse)
    for (int b = dc; b < n; ++b) D[b * n + b] = scale_moment(psi_c, it, itr) - m0r;
  for (int r = 0; r < dL; ++r) {
    R s = zero;
    for (int a = r; a < dc; ++a) s = r_fma(Li[a * n + r], scale_moment(M1[a], it, itr), s);
    g[r] = s;
  }
  R T[nn];
  for (int a = 0; a < dL; ++a)
    for (int c = 0; c < dL; ++c) {
      R s = zero;
      for (int b = c; b < dL; ++b) s = r_fma(D[a * n + b], Li[b * n + c], s);
      T[a * n + c] = s;
    }
  const R half = r_fromf<R>(0.5f);
  for (int r = 0; r < dL; ++r)
    for (int c = 0; c <= r; ++c) {
      R s = zero;
      for (int a = r; a < dL; ++a) s = r_fma(Li[a * n + r], T[a * n + c], s);
      G[r * n + c] = half * s;
      G[c * n + r] = half * s;
    }
  M0_out = m0;
  return true;
}

template <int n, typename QT, typename R>
PGV_BIG bool quad_all(const PlanDesc& P, int s, double& coll) {
  constexpr int nn = n * n;
  const int N = P.N;
  const R* mu = rp<R>(P.mu[s]);
  const R* Sd = rp<R>(P.Sd[s]);
  R* gg = rp<R>(P.g);
  R* GG = rp<R>(P.G);
  coll = 0.0;
  bool ok = true;
  for (int i = 0; i <= N; ++i) {
    R mu_i[n], S_ii[nn], g[n], G[nn];
    double m0;
    ld_vec<n, R>(mu + (size_t)i * n, mu_i);
    ld_blk<n, R>(Sd + (size_t)i * nn, S_ii);
    ok = quad_factor<n, QT, R>(P, i, mu_i, S_ii, g, G, m0) && ok;
    st_vec<n, R>(gg + (size_t)i * n, g);
    st_blk<n, R>(GG + (size_t)i * nn, G);
    coll += m0;
  }
  return ok;
}

// ------------------------------------------------------------ trial (a5)

struct TrialOut {
  double kl, logdet, prior_cost, delta, trace;
  bool pd;
};

// Thm 1 at step beta, scaled by s = beta+1:
//   A~ = beta (2G + K^-1) + Lambda_k          = (beta+1) Lambda'
//   M  = beta K^-1 + Lambda_k                 (mean system times beta)
//   M delta = beta (-g + b - K^-1 mu_k),      mu' = mu_k + delta
// The natural-gradient step (Sec. 3.1(d); P.update == PGVIMP_UPDATE_NGD) has
// the same form with s = 1, Lambda_k weighted by c = 1 - beta and M = A~:
//   A~ = beta (2G + K^-1) + (1 - beta) Lambda_k = Lambda',
//   Lambda' delta = beta (-g + b - K^-1 mu_k),
// the step of the natural parameters (Lambda mu, -Lambda/2) along minus the
// gradient in the expectation parameters.  One forward sweep eliminates A~ and
// M together (they share the off-diagonal blocks); one backward sweep produces
// Sigma~ = A~^-1 (selected blocks), delta and the KL pieces
//   KL = 1/2 [beta tr((Lambda_k - 2G - K^-1) Sigma~) + delta^T Lambda_k delta
//             + log det Lambda' - log det Lambda_k]
// (both updates: tr(Lambda_k Sigma') - D = tr((Lambda_k - Lambda') Sigma') =
// tr((s Lambda_k - A~) Sigma~)).  Results go to buffer set `out`: mu',
// Sigma' = s Sigma~.  Carried between states: the packed Schur terms of both
// eliminations, W^M_{i-1} y_{i-1} and K^-1_{i,i-1} mu_{i-1} (vectors), not the
// matrices.
template <int n, typename R>
PGV_BIG TrialOut trial(const PlanDesc& P, double beta_d, int cur, int out, double logdet_k) {
  constexpr int nn = n * n, np = Scr<n>::np, SS = Scr<n>::stride;
  const int N = P.N;
  const R* mu = rp<R>(P.mu[cur]);
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* Ld = rp<R>(P.Ld);
  const R* Lo = rp<R>(P.Lo);
  const R* GG = rp<R>(P.G);
  const R* gg = rp<R>(P.g);
  const R* bb = rp<R>(P.b);
  const R* mubar = rp<R>(P.mubar);
  R* scr = rp<R>(P.scr);
  TrialOut res;
  res.kl = INFINITY;
  res.pd = false;
  res.logdet = 0.0;
  res.prior_cost = 0.0;
  res.delta = 0.0;
  res.trace = 0.0;
  const R beta = r_from<R>(beta_d), beta2 = beta + beta, zero = r_fromf<R>(0.0f);
  const bool ngd = (P.update == PGVIMP_UPDATE_NGD);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);   // weight of Lambda_k
  R SA[np], SM[np], vM[n], q[n], mi[n];
#pragma unroll (n <= 8 ? 32 : 0)
  for (int e = 0; e < np; ++e) {
    SA[e] = zero;
    SM[e] = zero;
  }
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a) {
    vM[a] = zero;
    q[a] = zero;
  }
  ld_vec<n, R>(mu, mi);
  LogDetAcc<R> ldA, ldM;
  ldA.init();
  ldM.init();
  bool okA = true, okM = true;
  for (int i = 0; i <= N; ++i) {
    R CA[np], CM[np], Kmu[n];
    {
      R B[nn];
      ld_blk<n, R>(Kd + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) {
        R s = q[a];
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) s = r_fma(B[a * n + c], mi[c], s);
        Kmu[a] = s;
      }
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c <= a; ++c) {
          R kb = beta * B[a * n + c];
          CM[pk(a, c)] = kb - SM[pk(a, c)];
          CA[pk(a, c)] = kb - SA[pk(a, c)];
        }
      ld_blk<n, R>(GG + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c <= a; ++c) {
          CA[pk(a, c)] = r_fma(beta2, B[a * n + c], CA[pk(a, c)]);
          if (ngd) CM[pk(a, c)] = r_fma(beta2, B[a * n + c], CM[pk(a, c)]);
        }
      ld_blk<n, R>(Ld + (size_t)i * nn, B);
      if (ngd)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int e = 0; e < nn; ++e) B[e] = cL * B[e];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c <= a; ++c) {
          CA[pk(a, c)] = CA[pk(a, c)] + B[a * n + c];
          CM[pk(a, c)] = CM[pk(a, c)] + B[a * n + c];
        }
    }
    R CiA[np], CiM[np];
    chol_inverse<n, R>(CA, CiA, ldA, okA);
    chol_inverse<n, R>(CM, CiM, ldM, okM);
    R E[nn], mnext[n];
    if (i < N) {
      ld_vec<n, R>(mu + (size_t)(i + 1) * n, mnext);
      ld_blk<n, R>(Ko + (size_t)i * nn, E);
      // K^-1 mu at i gets K^-1_{i,i+1} mu_{i+1}; at i+1 it gets K^-1_{i+1,i} mu_i
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) {
        R s = zero, t = zero;
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          s = r_fma(E[c * n + a], mnext[c], s);
          t = r_fma(E[a * n + c], mi[c], t);
        }
        Kmu[a] = Kmu[a] + s;
        q[a] = t;
      }
      R B[nn];
      ld_blk<n, R>(Lo + (size_t)i * nn, B);
      if (ngd)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int e = 0; e < nn; ++e) B[e] = cL * B[e];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < nn; ++e) E[e] = r_fma(beta, E[e], B[e]);   // beta K^-1_{i+1,i} + c Lambda_{i+1,i}
    }
    R y[n], z[n];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) {
      R r = (bb[(size_t)i * n + a] - gg[(size_t)i * n + a]) - Kmu[a];
      y[a] = r_fma(beta, r, -vM[a]);
    }
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) {
      R s = CiM[pk(a, 0)] * y[0];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int c = 1; c < n; ++c) s = r_fma(CiM[pk(a, c)], y[c], s);
      z[a] = s;
    }
    R* sp = scr + (size_t)i * SS;
    st_packed<n, R>(sp + Scr<n>::oCi, CiA);
    st_vec<n, R>(sp + Scr<n>::oZ, z);
    if (i < N) {
      R W[nn];
      mul_full_sym<n, R>(E, CiA, W);
      mul_nt_packed<n, R>(W, E, SA);
      st_blk<n, R>(sp + Scr<n>::oWA, W);
      mul_full_sym<n, R>(E, CiM, W);
      mul_nt_packed<n, R>(W, E, SM);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) {
        R s = W[a * n] * y[0];
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 1; c < n; ++c) s = r_fma(W[a * n + c], y[c], s);
        vM[a] = s;
      }
      st_blk<n, R>(sp + Scr<n>::oWM, W);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) mi[a] = mnext[a];
    }
  }
  if (!okA || !okM) return res;
  res.pd = true;
  const double Dd = (double)n * (N + 1);
  const double bp1d = ngd ? 1.0 : beta_d + 1.0;        // s
  res.logdet = ldA.log_value() - (ngd ? 0.0 : Dd * log(bp1d));
  const R bp1 = r_from<R>(bp1d), mbp1 = -bp1;
  // backward sweep
  R* mo_out = rp<R>(P.mu[out]);
  R* Sd_out = rp<R>(P.Sd[out]);
  R* So_out = rp<R>(P.So[out]);
  R Sn[np], xn[n], dpn[n];
  R trc = zero, dl = zero, ktr = zero, kq = zero;
  {
    const R* sp = scr + (size_t)N * SS;
    ld_packed<n, R>(sp + Scr<n>::oCi, Sn);
    ld_vec<n, R>(sp + Scr<n>::oZ, xn);
    R B[nn], Lb[nn];
    ld_blk<n, R>(Ld + (size_t)N * nn, Lb);
    ld_blk<n, R>(GG + (size_t)N * nn, B);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) trc = r_fma(Lb[a * n + c] - (B[a * n + c] + B[a * n + c]), Sn[pk(a, c)], trc);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) dl = r_fma(xn[a] * Lb[a * n + c], xn[c], dl);
    ld_blk<n, R>(Kd + (size_t)N * nn, B);
    R mo[n];
    for (int a = 0; a < n; ++a) {
      mo[a] = mu[(size_t)N * n + a] + xn[a];
      dpn[a] = mo[a] - mubar[(size_t)N * n + a];
    }
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) {
        trc = r_fma(-B[a * n + c], Sn[pk(a, c)], trc);
        ktr = r_fma(B[a * n + c], Sn[pk(a, c)], ktr);
        kq = r_fma(dpn[a] * B[a * n + c], dpn[c], kq);
      }
    R Sfull[np];
    for (int e = 0; e < np; ++e) Sfull[e] = bp1 * Sn[e];
    st_sym<n, R>(Sd_out + (size_t)N * nn, Sfull);
    st_vec<n, R>(mo_out + (size_t)N * n, mo);
  }
  for (int i = N - 1; i >= 0; --i) {
    const R* sp = scr + (size_t)i * SS;
    R Si[np], T[nn], xi[n];
    {
      R W[nn], Ci[np];
      ld_blk<n, R>(sp + Scr<n>::oWA, W);
      ld_packed<n, R>(sp + Scr<n>::oCi, Ci);
      mul_sym_full<n, R>(Sn, W, T);            // T = Sigma~_{i+1} W_i = -Sigma~_{i+1,i}
      add_tn_packed<n, R>(Ci, W, T, Si);
    }
    {
      R WM[nn], z[n];
      ld_blk<n, R>(sp + Scr<n>::oWM, WM);
      ld_vec<n, R>(sp + Scr<n>::oZ, z);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) {
        R s = z[a];
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) s = r_fma(-WM[c * n + a], xn[c], s);
        xi[a] = s;
      }
    }
    R mo[n], dpi[n];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) {
      mo[a] = mu[(size_t)i * n + a] + xi[a];
      dpi[a] = mo[a] - mubar[(size_t)i * n + a];
    }
    {
      R B[nn];
      ld_blk<n, R>(Ld + (size_t)i * nn, B);    // Lambda_k: trace, delta^T Lambda_k delta
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          trc = r_fma(B[a * n + c], Si[pk(a, c)], trc);
          dl = r_fma(xi[a] * B[a * n + c], xi[c], dl);
        }
      ld_blk<n, R>(GG + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) trc = r_fma(-(B[a * n + c] + B[a * n + c]), Si[pk(a, c)], trc);
      ld_blk<n, R>(Kd + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          trc = r_fma(-B[a * n + c], Si[pk(a, c)], trc);
          ktr = r_fma(B[a * n + c], Si[pk(a, c)], ktr);
          kq = r_fma(dpi[a] * B[a * n + c], dpi[c], kq);
        }
      ld_blk<n, R>(Lo + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          trc = r_fma(-(B[a * n + c] + B[a * n + c]), T[a * n + c], trc);
          dl = r_fma((xn[a] + xn[a]) * B[a * n + c], xi[c], dl);
        }
      ld_blk<n, R>(Ko + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          trc = r_fma(B[a * n + c] + B[a * n + c], T[a * n + c], trc);
          ktr = r_fma(-(B[a * n + c] + B[a * n + c]), T[a * n + c], ktr);
          kq = r_fma((dpn[a] + dpn[a]) * B[a * n + c], dpi[c], kq);
        }
    }
    {
      R X[np];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < np; ++e) X[e] = bp1 * Si[e];
      st_sym<n, R>(Sd_out + (size_t)i * nn, X);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < nn; ++e) T[e] = mbp1 * T[e];
      st_blk<n, R>(So_out + (size_t)i * nn, T);
      st_vec<n, R>(mo_out + (size_t)i * n, mo);
    }
#pragma unroll (n <= 8 ? 32 : 0)
    for (int e = 0; e < np; ++e) Sn[e] = Si[e];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) {
      xn[a] = xi[a];
      dpn[a] = dpi[a];
    }
  }
  res.trace = beta_d * r_to(trc);
  res.delta = r_to(dl);
  res.kl = 0.5 * (res.trace + res.delta + res.logdet - logdet_k);
  res.prior_cost = 0.5 * (bp1d * r_to(ktr) + r_to(kq));
  return res;
}

// Two-phase temperature: when the plan reaches iteration switch_iter with a
// prior still at the low temperature, K^-1 and b (built with 1/T_low) are
// scaled by T_low/T_high -- the prior rebuilt at T_high -- and so is the prior
// cost of the current iterate; mu_bar = K b does not change.  States i =
// first, first + stride, ... (all of them for one thread).
PGV_DEV bool temp_switch_due(const PlanDesc& P) {
  return P.inv_temp_high > 0.0 && P.scal[S_K] >= (double)P.switch_iter && P.scal[S_THIGH] == 0.0;
}
template <int n, typename R>
PGV_BIG void switch_temperature(const PlanDesc& P, int first, int stride) {
  constexpr int nn = n * n;
  const int N = P.N;
  const R f = r_from<R>(P.inv_temp_high / P.inv_temp);
  R* Kd = rp<R>(P.Kd);
  R* Ko = rp<R>(P.Ko);
  R* b = rp<R>(P.b);
  for (int i = first; i <= N; i += stride) {
    for (int e = 0; e < nn; ++e) Kd[(size_t)i * nn + e] = f * Kd[(size_t)i * nn + e];
    if (i < N)
      for (int e = 0; e < nn; ++e) Ko[(size_t)i * nn + e] = f * Ko[(size_t)i * nn + e];
    for (int a = 0; a < n; ++a) b[(size_t)i * n + a] = f * b[(size_t)i * n + a];
  }
  if (first == 0) {   // done by one thread; block callers synchronise before reading it
    P.scal[S_PRIOR] = P.scal[S_PRIOR] * (P.inv_temp_high / P.inv_temp);
    P.scal[S_THIGH] = 1.0;
  }
}

// Lambda_{k+1} = A~(beta) / s, written over (Ld, Lo): s = beta+1 (Thm 1) or
// 1 with Lambda_k weighted by 1 - beta (natural-gradient step).
template <int n, typename R>
PGV_BIG void accept_precision(const PlanDesc& P, double beta_d) {
  constexpr int nn = n * n;
  const int N = P.N;
  const bool ngd = (P.update == PGVIMP_UPDATE_NGD);
  const R inv = r_from<R>(ngd ? 1.0 : 1.0 / (beta_d + 1.0)), beta = r_from<R>(beta_d), two = r_fromf<R>(2.0f);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);
  R* Ld = rp<R>(P.Ld);
  R* Lo = rp<R>(P.Lo);
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* GG = rp<R>(P.G);
  for (int i = 0; i <= N; ++i) {
    R K[nn], Lb[nn], Gb[nn];
    ld_blk<n, R>(Kd + (size_t)i * nn, K);
    ld_blk<n, R>(Ld + (size_t)i * nn, Lb);
    ld_blk<n, R>(GG + (size_t)i * nn, Gb);
#pragma unroll (n <= 8 ? 32 : 0)
    for (int e = 0; e < nn; ++e) Lb[e] = r_fma(beta, r_fma(two, Gb[e], K[e]), cL * Lb[e]) * inv;
    st_blk<n, R>(Ld + (size_t)i * nn, Lb);
    if (i < N) {
      ld_blk<n, R>(Ko + (size_t)i * nn, K);
      ld_blk<n, R>(Lo + (size_t)i * nn, Lb);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < nn; ++e) Lb[e] = r_fma(beta, K[e], cL * Lb[e]) * inv;
      st_blk<n, R>(Lo + (size_t)i * nn, Lb);
    }
  }
}

// One proximal iteration (Alg. 1 loop body): quadrature and gradients at the
// current iterate, the largest feasible step by bisection (App. C: beta_max
// first, then max_bisect halvings of [0, beta_max]; feasible = Lambda'
// positive definite and KL <= eps, decided in FP64), and the update.
template <int n, typename QT, typename R>
PGV_BIG void iterate_once(const PlanDesc& P) {
  double* sc = P.scal;
  if (temp_switch_due(P)) switch_temperature<n, R>(P, 0, 1);
  const int cur = (int)sc[S_CUR];
  const int oa = (cur + 1) % 3, ob = (cur + 2) % 3;
  double coll;
  if (!quad_all<n, QT, R>(P, cur, coll)) {
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
  double beta = P.beta_max, lo = 0.0, hi = P.beta_max;
  int into = oa, halvings = 0;
  bool searching = false;
  for (;;) {
    TrialOut Rt = trial<n, R>(P, beta, cur, into, logdet_k);
    ++trials;
    if (Rt.pd && has_eps) margin = fmin(margin, fabs(Rt.kl - eps) / eps);
    const bool feas = Rt.pd && (Rt.kl <= eps);
    if (feas) {
      best = into;
      best_beta = beta;
      bestR = Rt;
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
    accept_precision<n, R>(P, best_beta);
    sc[S_CUR] = (double)best;
    sc[S_LOGDET] = bestR.logdet;
    sc[S_PRIOR] = bestR.prior_cost;
  }
  sc[S_COLL] = coll;
  sc[S_K] = (double)(k + 1);
  sc[S_KIN] = sc[S_KIN] + 1.0;
}

// Initial iterate (mu_0 on the straight line in q with constant qdot;
// Lambda_0 = K^-1 or init_scale * I) and its marginals.
template <int n, typename R>
PGV_BIG void init_plan(const PlanDesc& P) {
  constexpr int nn = n * n;
  double* sc = P.scal;
  const int N = P.N, nq = P.nq;
  R* mu0 = rp<R>(P.mu[0]);
  for (int i = 0; i <= N; ++i) {
    double s = (double)i / N;
    for (int a = 0; a < nq; ++a) {
      double d = P.muN[a] - P.mu0[a];
      mu0[(size_t)i * n + a] = r_from<R>(P.mu0[a] + s * d);
      mu0[(size_t)i * n + nq + a] = r_from<R>(d / P.T);
    }
  }
  R* Ld = rp<R>(P.Ld);
  R* Lo = rp<R>(P.Lo);
  const R zero = r_fromf<R>(0.0f), sI = r_from<R>(P.init_scale);
  for (int i = 0; i <= N; ++i) {
    R blk[nn];
    if (P.init_kind == 1) {
      for (int e = 0; e < nn; ++e) blk[e] = zero;
      for (int a = 0; a < n; ++a) blk[a * n + a] = sI;
    } else {
      ld_blk<n, R>(rp<R>(P.Kd) + (size_t)i * nn, blk);
    }
    st_blk<n, R>(Ld + (size_t)i * nn, blk);
    if (i < N) {
      if (P.init_kind == 1)
        for (int e = 0; e < nn; ++e) blk[e] = zero;
      else
        ld_blk<n, R>(rp<R>(P.Ko) + (size_t)i * nn, blk);
      st_blk<n, R>(Lo + (size_t)i * nn, blk);
    }
  }
  double ld, pc;
  if (!marginals<n, R>(P, 0, ld, pc)) {
    sc[S_STATUS] = 2.0;
    return;
  }
  sc[S_CUR] = 0.0;
  sc[S_LOGDET] = ld;
  sc[S_PRIOR] = pc;
  sc[S_K] = 0.0;
  sc[S_KIN] = 0.0;
  sc[S_INIT] = 1.0;
  sc[S_FMT] = 0.0;
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
  if (P.rule == PGVIMP_RULE_SMOLYAK) {
    for (int l = 0; l < P.sgs_rows; ++l) {
      const double* row = P.sgs + (size_t)l * (n + 1);
      QT xi[n];
      for (int a = 0; a < n; ++a) xi[a] = (QT)row[a];
      accum(xi, (QT)row[n]);
    }
  } else if (P.rule == PGVIMP_RULE_DEG3) {
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
    QT xq[kMaxGH], wq[kMaxGH];   // the 1-D rule, converted once
    for (int d = 0; d < p; ++d) {
      xq[d] = (QT)P.gh_x[p * kMaxGH + d];
      wq[d] = (QT)P.gh_w[p * kMaxGH + d];
    }
    for (int l = 0; l < Pn; ++l) {
      QT xi[n];
      QT w = 1;
      int rem = l;
      for (int a = n - 1; a >= 0; --a) {
        int d = rem % p;
        rem /= p;
        xi[a] = xq[d];
        w *= wq[d];
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

template <int n, typename QT, typename R>
PGV_BIG bool slr_all(const PlanDesc& P, bool first) {
  constexpr int nn = n * n;
  const int N = P.N, nq = P.nq;
  double xb[n], Sb[nn];
  bool ok = true;
  const int cur = (int)P.scal[S_CUR];
  const R* mu = rp<R>(P.mu[cur]);
  const R* Sd = rp<R>(P.Sd[cur]);
  for (int i = 0; i <= N; ++i) {
    if (first) {
      double s = (double)i / N;
      for (int a = 0; a < nq; ++a) {
        double d = P.muN[a] - P.mu0[a];
        xb[a] = P.mu0[a] + s * d;
        xb[nq + a] = d / P.T;
      }
      for (int e = 0; e < nn; ++e) Sb[e] = P.K0[e];
    } else {
      for (int a = 0; a < n; ++a) xb[a] = r_to(mu[(size_t)i * n + a]);
      for (int e = 0; e < nn; ++e) Sb[e] = r_to(Sd[(size_t)i * nn + e]);
    }
    for (int a = 0; a < n; ++a) P.xbar[(size_t)i * n + a] = xb[a];
    if (i < N) ok = slr_step<n, QT>(P, xb, Sb, P.Altv + (size_t)i * nn, P.altv + (size_t)i * n) && ok;
  }
  return ok;
}

// ------------------------------------------------------------ kernels

#define PLAN_OR_RETURN                                     \
  const int t = blockIdx.x * blockDim.x + threadIdx.x;     \
  if (t >= count) return;                                  \
  const PlanDesc& P = descs[t];

// Prior build; `mode` 0: linear system (A, a); 1: the SLR linearisation.
template <int n, typename R>
__global__ void k_prior(const PlanDesc* __restrict__ descs, int count, int mode) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  if (!prior_build<n, R>(P, mode == 1)) P.scal[S_STATUS] = 1.0;
}

template <int n, typename R>
__global__ void k_init(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  init_plan<n, R>(P);
}

// After a relinearisation: the prior cost of the current iterate under the
// new prior, and a fresh inner-iteration counter.
template <int n, typename R>
__global__ void k_relinearised(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  P.scal[S_PRIOR] = prior_cost_of<n, R>(P, (int)P.scal[S_CUR]);
  P.scal[S_KIN] = 0.0;
}

// Occupancy of the fused iterations: for n = 4 a cap of 128 registers per
// thread (16 warps per SM; the block arrays spill a little to L1) measured 16%
// more plans/s than 255 registers at 8 warps per SM on B300 with double-float
// recursions, 3% with FP64 recursions; 80 registers (24 warps) spilled more
// and lost.  Larger n keep the full register file.
template <int n>
constexpr int iter_min_blocks() { return n == 4 ? 8 : 1; }

template <int n, typename QT, typename R>
__global__ void __launch_bounds__(64, iter_min_blocks<n>()) k_iterate(const PlanDesc* __restrict__ descs, int count,
                                                                     int iters) {
  PLAN_OR_RETURN
  for (int it = 0; it < iters; ++it) {
    if (P.scal[S_STATUS] != 0.0 || P.scal[S_INIT] == 0.0) return;
    if ((int)P.scal[S_KIN] >= P.iters) return;
    iterate_once<n, QT, R>(P);
  }
}

template <int n, typename R>
PGV_DEV double slr_norm(const PlanDesc& P) {
  const int cur = (int)P.scal[S_CUR];
  const R* mu = rp<R>(P.mu[cur]);
  double s = 0.0;
  for (size_t e = 0; e < (size_t)(P.N + 1) * n; ++e) {
    double d = r_to(mu[e]) - P.xbar[e];
    s = fma(d, d, s);
  }
  return sqrt(s);
}

// SLR linearisation.  mode 1: the straight-line nominal with K0 (first outer
// iteration); 0: the current iterate, closing the previous outer iteration
// (its norm); 2: the current iterate without bookkeeping.
template <int n, typename QT, typename R>
__global__ void k_slr(const PlanDesc* __restrict__ descs, int count, int mode) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  if (mode == 0) {
    const int j = (int)P.scal[S_J];
    if (j < P.slr_iters) P.slr_norms[j] = slr_norm<n, R>(P);
    P.scal[S_J] = (double)(j + 1);
  }
  if (!slr_all<n, QT, R>(P, mode == 1)) P.scal[S_STATUS] = 4.0;
}

// Final SLR norm after the last linearisation's iterations.
template <int n, typename R>
__global__ void k_slr_finish(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  if (P.scal[S_STATUS] != 0.0) return;
  const int j = (int)P.scal[S_J];
  if (j < P.slr_iters) P.slr_norms[j] = slr_norm<n, R>(P);
  P.scal[S_J] = (double)(j + 1);
}

// Moves the current iterate into buffer set 0 (the one results are read
// from); with double-float storage also converts the result buffers (set 0,
// Lambda) to FP64 in place.  k_working undoes that conversion.
template <int n, typename R>
__global__ void k_finalize(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  const int cur = (int)P.scal[S_CUR];
  const size_t N = P.N;
  if (cur != 0 && P.scal[S_FMT] == 0.0) {
    R* m0 = rp<R>(P.mu[0]);
    R* s0 = rp<R>(P.Sd[0]);
    R* o0 = rp<R>(P.So[0]);
    const R* mc = rp<R>(P.mu[cur]);
    const R* sc = rp<R>(P.Sd[cur]);
    const R* oc = rp<R>(P.So[cur]);
    for (size_t e = 0; e < (N + 1) * n; ++e) m0[e] = mc[e];
    for (size_t e = 0; e < (N + 1) * n * n; ++e) s0[e] = sc[e];
    for (size_t e = 0; e < N * n * n; ++e) o0[e] = oc[e];
    P.scal[S_CUR] = 0.0;
  }
  if (!std::is_same<R, double>::value && P.scal[S_FMT] == 0.0) {
    double* bufs[5] = {P.mu[0], P.Sd[0], P.So[0], P.Ld, P.Lo};
    const size_t cnt[5] = {(N + 1) * n, (N + 1) * n * n, N * n * n, (N + 1) * n * n, N * n * n};
    for (int k = 0; k < 5; ++k) {
      R* rbuf = rp<R>(bufs[k]);
      for (size_t e = 0; e < cnt[k]; ++e) {
        double v = r_to(rbuf[e]);
        bufs[k][e] = v;
      }
    }
    P.scal[S_FMT] = 1.0;
  }
}

template <int n, typename R>
__global__ void k_working(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  const size_t N = P.N;
  if (!std::is_same<R, double>::value && P.scal[S_FMT] == 1.0) {
    double* bufs[5] = {P.mu[0], P.Sd[0], P.So[0], P.Ld, P.Lo};
    const size_t cnt[5] = {(N + 1) * n, (N + 1) * n * n, N * n * n, (N + 1) * n * n, N * n * n};
    for (int k = 0; k < 5; ++k) {
      R* rbuf = rp<R>(bufs[k]);
      for (size_t e = 0; e < cnt[k]; ++e) {
        R v = r_from<R>(bufs[k][e]);
        rbuf[e] = v;
      }
    }
    P.scal[S_FMT] = 0.0;
  }
}

// Single-row phases (per-row checks through the C ABI), FP64 recursions.
template <int n>
__global__ void k_marginals(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  double ld, pc;
  const int cur = (int)P.scal[S_CUR];
  bool ok = marginals<n, double>(P, cur, ld, pc);
  P.scal[S_LOGDET] = ld;
  P.scal[S_PRIOR] = pc;
  if (!ok) P.scal[S_STATUS] = 2.0;
}

template <int n, typename QT>
__global__ void k_quad(const PlanDesc* __restrict__ descs, int count) {
  PLAN_OR_RETURN
  double coll;
  bool ok = quad_all<n, QT, double>(P, (int)P.scal[S_CUR], coll);
  P.scal[S_COLL] = coll;
  if (!ok) P.scal[S_STATUS] = 3.0;
}

template <int n>
__global__ void k_trial(const PlanDesc* __restrict__ descs, int count, double beta) {
  PLAN_OR_RETURN
  const int cur = (int)P.scal[S_CUR];
  TrialOut R = trial<n, double>(P, beta, cur, (cur + 2) % 3, P.scal[S_LOGDET]);
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
//   iter<n, QT, R>: the fused proximal iterations (Alg. 1 loop);
//   aux<n, R>:      prior build, initial iterate, SLR, bookkeeping kernels;
//   rows<n>:        the single-row kernels (marginals, quadrature, one trial).
enum { PH_PRIOR = 100, PH_INIT = 101, PH_ITER = 102, PH_SLR = 103, PH_RELIN = 104, PH_SLR_FIN = 105,
       PH_FINALIZE = 106, PH_WORKING = 107 };

template <int n, typename QT, typename R>
cudaError_t launch_iter(const Launch& L, int iters) {
  const int tpb = 32;
  k_iterate<n, QT, R><<<blocks_for(L.count, tpb), tpb, 0, L.stream>>>(L.descs, L.count, iters);
  return cudaGetLastError();
}

// `qt32`: FP32 quadrature in the SLR kernel.
template <int n, typename R>
cudaError_t launch_aux(const Launch& L, int phase, int arg_i, int qt32) {
  const int tpb = 32;
  dim3 g(blocks_for(L.count, tpb)), b(tpb);
  switch (phase) {
    case PH_PRIOR: k_prior<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i); break;
    case PH_INIT: k_init<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_SLR:
      if (qt32) k_slr<n, float, R><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i);
      else k_slr<n, double, R><<<g, b, 0, L.stream>>>(L.descs, L.count, arg_i);
      break;
    case PH_RELIN: k_relinearised<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_SLR_FIN: k_slr_finish<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_FINALIZE: k_finalize<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
    case PH_WORKING: k_working<n, R><<<g, b, 0, L.stream>>>(L.descs, L.count); break;
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
