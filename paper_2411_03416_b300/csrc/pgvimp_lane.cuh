// pgvimp_lane.cuh -- the lane form of the fused iteration for state dimension
// n = 4: sixteen lanes (half a warp) own one plan, lane l = 4a + c holding
// element (a, c) of every 4 x 4 block the sweeps touch.
//
// Why: in the thread form one thread runs a whole plan, so each warp load
// touches 32 plans' memory (32 separate sectors) and every block operation
// is unrolled straight-line code; with double-float arithmetic one state step
// of a trial is ~190 KB of instructions, far beyond the instruction cache, and
// warps stall on instruction fetch and on uncoalesced loads.  Here a block of
// one state is one coalesced 128-byte access by sixteen lanes, the per-state
// body is a few KB (each lane does n FMAs per block product, with operands
// exchanged by shuffles), and the next state's blocks are prefetched into
// registers (one element per lane) while the current state is eliminated.
//
// The arithmetic is that of `trial` / `iterate_once` in pgvimp_kernels.cuh
// (Thm 1 and the natural-gradient step; App. C step-size search decided in
// FP64 from the same quantities), with two differences of order: the 4 x 4
// pivot blocks are inverted by Gauss-Jordan elimination without pivoting (the
// pivots are the Cholesky pivots of the same SPD block, so positive
// definiteness and log det are decided from the same Schur complements), and
// sums over a block row are formed by a butterfly of shuffles.  Vectors over
// a block row (y, z, the mean correction) are held replicated in the four
// lanes of the row.  The quadrature (Sec. 4.3) runs one state per lane with
// the thread form's quad_factor.
#pragma once
#include "pgvimp_dfx.cuh"
#include "pgvimp_kernels.cuh"

namespace pgv {
namespace lanef {

constexpr int kN = 4, kNN = 16;
// Per-state scratch (R elements): Ci of A~ (full, element l), W_A, W_M, z.
constexpr int oCi = 0, oWA = 16, oWM = 32, oZ = 48, kStride = 52;   // = 3 n^2 + n

struct Lane {
  unsigned mask;   // the sixteen lanes of this plan
  int base;        // 0 or 16
  int l, a, c;     // element index l = 4a + c
};

PGV_DEV Lane make_lane() {
  Lane x;
  const int lane = threadIdx.x & 31;
  x.base = lane & 16;
  x.mask = 0xffffu << x.base;
  x.l = lane & 15;
  x.a = x.l >> 2;
  x.c = x.l & 3;
  return x;
}

// Value held by lane `src` (0..15) of this plan.
PGV_DEV double sh(const Lane& x, double v, int src) { return __shfl_sync(x.mask, v, x.base + src); }
PGV_DEV float sh(const Lane& x, float v, int src) { return __shfl_sync(x.mask, v, x.base + src); }
PGV_DEV df64 sh(const Lane& x, df64 v, int src) {
  return df_make(__shfl_sync(x.mask, v.hi, x.base + src), __shfl_sync(x.mask, v.lo, x.base + src));
}
PGV_DEV double shx(const Lane& x, double v, int m) { return __shfl_xor_sync(x.mask, v, m); }
PGV_DEV df64 shx(const Lane& x, df64 v, int m) {
  return df_make(__shfl_xor_sync(x.mask, v.hi, m), __shfl_xor_sync(x.mask, v.lo, m));
}
// Sum over the four lanes of a block row (every lane of the row gets the same
// value: the butterfly pairs the same operands in every lane and + commutes).
template <typename R>
PGV_DEV R rowsum(const Lane& x, R v) {
  v = v + shx(x, v, 1);
  return v + shx(x, v, 2);
}
// Sum over the sixteen lanes.
template <typename R>
PGV_DEV R halfsum(const Lane& x, R v) {
  v = v + shx(x, v, 1);
  v = v + shx(x, v, 2);
  v = v + shx(x, v, 4);
  return v + shx(x, v, 8);
}
PGV_DEV double halfsum_d(const Lane& x, double v) {
  v += shx(x, v, 1);
  v += shx(x, v, 2);
  v += shx(x, v, 4);
  return v + shx(x, v, 8);
}

// Cache hint: the line holding p, fetched into L1 ahead of its use (no
// register is held for it).
PGV_DEV void prefetch_l1(const void* p) { asm volatile("prefetch.L1 [%0];" ::"l"(p)); }
// 2 v, exactly.
PGV_DEV double twice(double v) { return v + v; }
PGV_DEV df64 twice(df64 v) { return df_make(v.hi + v.hi, v.lo + v.lo); }

// 1/v.  FP64: Newton-Raphson on the hardware's approximate FP64 reciprocal
// (rcp.approx.ftz.f64, about 20 correct bits), two steps r + r (1 - v r) with
// FMA residuals, each doubling the correct bits, so the result is within a few
// ulp of 1/v; it replaces an IEEE division, whose FP64 instruction sequence
// took about half of the kernel's FP64 pipe.  Pivots below the normal range
// (the approximation flushes them) take the division.  Double-float: df_rcp.
PGV_DEV double r_rcp(double v) {
  if (!(v >= 2.2250738585072014e-308)) return 1.0 / v;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(v));
  double e = fma(-v, r, 1.0);
  r = fma(r, e, r);
  e = fma(-v, r, 1.0);
  return fma(r, e, r);
}
PGV_DEV df64 r_rcp(df64 v) { return df_rcp(v); }

// Four-term dot product sum_t x_t y_t: an FMA chain in FP64; the
// compensated double-float dot product df_dot4 otherwise (shorter and with
// more independent operations than four chained double-float FMAs).
PGV_DEV double dot4(const double* x, const double* y) {
  double s = x[0] * y[0];
#pragma unroll
  for (int t = 1; t < kN; ++t) s = fma(x[t], y[t], s);
  return s;
}
PGV_DEV df64 dot4(const df64* x, const df64* y) { return df_dot4(x, y); }

// (X Y)_{ac} = sum_t X_{at} Y_{tc}
template <typename R>
PGV_DEV R mm(const Lane& x, R X, R Y) {
  R u[kN], v[kN];
#pragma unroll
  for (int t = 0; t < kN; ++t) {
    u[t] = sh(x, X, 4 * x.a + t);
    v[t] = sh(x, Y, 4 * t + x.c);
  }
  return dot4(u, v);
}
// (X Y^T)_{ac} = sum_t X_{at} Y_{ct}
template <typename R>
PGV_DEV R mm_nt(const Lane& x, R X, R Y) {
  R u[kN], v[kN];
#pragma unroll
  for (int t = 0; t < kN; ++t) {
    u[t] = sh(x, X, 4 * x.a + t);
    v[t] = sh(x, Y, 4 * x.c + t);
  }
  return dot4(u, v);
}
// (X^T Y)_{ac} = sum_t X_{ta} Y_{tc}
template <typename R>
PGV_DEV R mm_tn(const Lane& x, R X, R Y) {
  R u[kN], v[kN];
#pragma unroll
  for (int t = 0; t < kN; ++t) {
    u[t] = sh(x, X, 4 * t + x.a);
    v[t] = sh(x, Y, 4 * t + x.c);
  }
  return dot4(u, v);
}

// In-place Gauss-Jordan inverses of the two symmetric positive definite
// blocks A and M of a state, held one element per lane, eliminated together
// (independent operations interleave) in a rolled loop over the pivots.  Step
// k divides by the pivot p_k, the k-th Schur complement's leading entry (the
// square of the k-th Cholesky diagonal), so `okA`/`okM` (all p_k > 0) and `ld`
// (the product of A's pivots; M's log det is not needed) are the Cholesky
// decisions.  The results are taken from the lower triangle, so they are
// exactly symmetric.
template <typename R>
PGV_DEV void gj_step(const Lane& x, int k, R& m, R p) {
  const R mkc = sh(x, m, 4 * k + x.c);
  const R mak = sh(x, m, 4 * x.a + k);
  const R ip = r_rcp(p);
  const R t = mkc * ip;
  const R u = mak * ip;
  const R upd = r_fma(-mak, t, m);
  m = (x.a == k) ? ((x.c == k) ? ip : t) : ((x.c == k) ? -u : upd);
}
template <typename R>
PGV_DEV void gj_inverse2(const Lane& x, R& A, R& M, LogDetAcc<R>& ld, bool& okA, bool& okM) {
  const R one = r_fromf<R>(1.0f);
#pragma unroll 1
  for (int k = 0; k < kN; ++k) {
    const R pa = sh(x, A, 5 * k);
    const R pm = sh(x, M, 5 * k);
    okA = okA && r_pos(pa);
    okM = okM && r_pos(pm);
    const R psa = r_pos(pa) ? pa : one;
    ld.mul(psa);
    gj_step(x, k, A, psa);
    gj_step(x, k, M, r_pos(pm) ? pm : one);
  }
  const R at = sh(x, A, 4 * x.c + x.a);
  const R mt = sh(x, M, 4 * x.c + x.a);
  if (x.a < x.c) {
    A = at;
    M = mt;
  }
}

// Thm 1 (or the natural-gradient step) at step beta, as `trial`: forward
// elimination of A~ and M with the mean right-hand side, backward selected
// inverse, mean correction and KL pieces.  Every lane of the plan returns the
// same TrialOut.
template <typename R>
PGV_BIG TrialOut trial_lane(const Lane& x, const PlanDesc& P, double beta_d, int cur, int out, double logdet_k) {
  const int N = P.N, l = x.l, a = x.a, c = x.c;
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
  const bool ngd = (P.update == PGVIMP_UPDATE_NGD);
  const R beta = r_from<R>(beta_d), zero = r_fromf<R>(0.0f);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);   // weight of Lambda_k

  // ---- forward: eliminate A~ and M, state by state; the lines of state
  // i+1's operands are fetched into L1 while state i is eliminated
  R SA = zero, SM = zero, vM = zero, q = zero;
  R mi_c = mu[c];
  LogDetAcc<R> ldA;
  ldA.init();
  bool okA = true, okM = true;
  for (int i = 0; i <= N; ++i) {
    const size_t o = (size_t)i * kNN;
    if (i < N) {
      const size_t o1 = o + kNN;
      prefetch_l1(Kd + o1 + l);
      prefetch_l1(GG + o1 + l);
      prefetch_l1(Ld + o1 + l);
      prefetch_l1(bb + (size_t)(i + 1) * kN + a);
      prefetch_l1(gg + (size_t)(i + 1) * kN + a);
      if (i + 1 < N) {
        prefetch_l1(Ko + o1 + l);
        prefetch_l1(Lo + o1 + l);
        prefetch_l1(mu + (size_t)(i + 2) * kN + c);
      }
    }
    const R K = Kd[o + l], G2 = twice(GG[o + l]), L = Ld[o + l];
    const R Lw = ngd ? cL * L : L;
    const R kb = beta * K;
    R CA = r_fma(beta, G2, kb + Lw) - SA;
    R CM = (ngd ? r_fma(beta, G2, kb + Lw) : kb + Lw) - SM;
    R Kmu = rowsum(x, K * mi_c) + q;               // (K^-1 mu_k)_i, row-replicated
    R CiA = CA, CiM = CM;
    gj_inverse2(x, CiA, CiM, ldA, okA, okM);
    R E = zero, mn_c = zero;
    if (i < N) {
      const R Eo = Ko[o + l], EoT = Ko[o + 4 * c + a], Lb = Lo[o + l];
      mn_c = mu[(size_t)(i + 1) * kN + c];
      Kmu = Kmu + rowsum(x, EoT * mn_c);            // + K^-1_{i,i+1} mu_{i+1}
      q = rowsum(x, Eo * mi_c);                     // K^-1_{i+1,i} mu_i, for state i+1
      E = r_fma(beta, Eo, ngd ? cL * Lb : Lb);      // beta K^-1_{i+1,i} + c Lambda_{i+1,i}
    }
    const R bg = bb[(size_t)i * kN + a] - gg[(size_t)i * kN + a];
    const R y = r_fma(beta, bg - Kmu, -vM);         // rhs of the reduced mean system
    const R y_c = sh(x, y, 4 * c + a);              // y_c in lane (a, c)
    const R z = rowsum(x, CiM * y_c);
    R* sp = scr + (size_t)i * kStride;
    sp[oCi + l] = CiA;
    if (c == 0) sp[oZ + a] = z;
    if (i < N) {
      const R WA = mm(x, E, CiA);
      const R WM = mm(x, E, CiM);
      SA = mm_nt(x, WA, E);
      SM = mm_nt(x, WM, E);
      vM = rowsum(x, WM * y_c);
      sp[oWA + l] = WA;
      sp[oWM + l] = WM;
    }
    mi_c = mn_c;
  }
  __syncwarp(x.mask);
  if (!okA || !okM) return res;
  res.pd = true;
  const double Dd = (double)kN * (N + 1);
  const double sd = ngd ? 1.0 : beta_d + 1.0;
  res.logdet = ldA.log_value() - (ngd ? 0.0 : Dd * log(sd));
  const R s = r_from<R>(sd), ms = -s;

  // ---- backward: selected inverse Sigma~ = A~^-1, mean correction, KL pieces
  R* mo_out = rp<R>(P.mu[out]);
  R* Sd_out = rp<R>(P.Sd[out]);
  R* So_out = rp<R>(P.So[out]);
  R trc = zero, dl = zero, ktr = zero, kq = zero;   // per-lane partial sums (element l)
  R Sn, xn, dpn;
  {
    const R* sp = scr + (size_t)N * kStride;
    Sn = sp[oCi + l];
    xn = sp[oZ + a];
    const size_t o = (size_t)N * kNN;
    const R Lk = Ld[o + l], Gk = GG[o + l], Kk = Kd[o + l];
    const R xn_c = sh(x, xn, 4 * c + a);
    const R mo = mu[(size_t)N * kN + a] + xn;
    dpn = mo - mubar[(size_t)N * kN + a];
    const R dpn_c = sh(x, dpn, 4 * c + a);
    trc = r_fma(Lk - twice(Gk) - Kk, Sn, trc);
    dl = r_fma(xn * Lk, xn_c, dl);
    ktr = r_fma(Kk, Sn, ktr);
    kq = r_fma(dpn * Kk, dpn_c, kq);
    Sd_out[o + l] = s * Sn;
    if (c == 0) mo_out[(size_t)N * kN + a] = mo;
  }
  for (int i = N - 1; i >= 0; --i) {
    if (i > 0) {   // the lines of state i-1's operands, fetched into L1 ahead of use
      const R* sp1 = scr + (size_t)(i - 1) * kStride;
      const size_t o1 = (size_t)(i - 1) * kNN;
      prefetch_l1(sp1 + oWA + l);
      prefetch_l1(sp1 + oCi + l);
      prefetch_l1(sp1 + oWM + l);
      prefetch_l1(sp1 + oZ + a);
      prefetch_l1(Ld + o1 + l);
      prefetch_l1(GG + o1 + l);
      prefetch_l1(Kd + o1 + l);
      prefetch_l1(Lo + o1 + l);
      prefetch_l1(Ko + o1 + l);
      prefetch_l1(mu + (size_t)(i - 1) * kN + a);
      prefetch_l1(mubar + (size_t)(i - 1) * kN + a);
    }
    const R* sp = scr + (size_t)i * kStride;
    const size_t oi = (size_t)i * kNN;
    const R W = sp[oWA + l], Ci = sp[oCi + l], WMT = sp[oWM + 4 * c + a], z = sp[oZ + a];
    const R Lk = Ld[oi + l], Gk = GG[oi + l], Kk = Kd[oi + l], Lob = Lo[oi + l], Kob = Ko[oi + l];
    const R mui = mu[(size_t)i * kN + a], mbi = mubar[(size_t)i * kN + a];
    const R T = mm(x, Sn, W);                      // Sigma~_{i+1} W_i = -Sigma~_{i+1,i}
    const R Si = Ci + mm_tn(x, W, T);              // C_i^-1 + W_i^T Sigma~_{i+1} W_i
    const R xn_c = sh(x, xn, 4 * c + a);
    const R xi = z - rowsum(x, WMT * xn_c);        // z_i - W^M_i^T x_{i+1}
    const R mo = mui + xi;
    const R dpi = mo - mbi;
    const R xi_c = sh(x, xi, 4 * c + a);
    const R dpi_c = sh(x, dpi, 4 * c + a);
    const R Ko2 = twice(Kob);
    trc = r_fma(Lk - twice(Gk) - Kk, Si, trc);
    trc = r_fma(Ko2 - twice(Lob), T, trc);
    dl = r_fma(xi * Lk, xi_c, dl);
    dl = r_fma(twice(xn) * Lob, xi_c, dl);
    ktr = r_fma(Kk, Si, ktr);
    ktr = r_fma(-Ko2, T, ktr);
    kq = r_fma(dpi * Kk, dpi_c, kq);
    kq = r_fma(twice(dpn) * Kob, dpi_c, kq);
    const size_t o = (size_t)i * kNN;
    Sd_out[o + l] = s * Si;
    So_out[o + l] = ms * T;
    if (c == 0) mo_out[(size_t)i * kN + a] = mo;
    Sn = Si;
    xn = xi;
    dpn = dpi;
  }
  const double trc_t = halfsum_d(x, r_to(trc)), dl_t = halfsum_d(x, r_to(dl));
  const double ktr_t = halfsum_d(x, r_to(ktr)), kq_t = halfsum_d(x, r_to(kq));
  res.trace = beta_d * trc_t;
  res.delta = dl_t;
  res.kl = 0.5 * (res.trace + res.delta + res.logdet - logdet_k);
  res.prior_cost = 0.5 * (sd * ktr_t + kq_t);
  return res;
}

// Lambda_{k+1} = A~(beta) / s over (Ld, Lo), one block per step of the
// sixteen lanes.
template <typename R>
PGV_BIG void accept_lane(const Lane& x, const PlanDesc& P, double beta_d) {
  const int N = P.N, l = x.l;
  const bool ngd = (P.update == PGVIMP_UPDATE_NGD);
  const R inv = r_from<R>(ngd ? 1.0 : 1.0 / (beta_d + 1.0)), beta = r_from<R>(beta_d), two = r_fromf<R>(2.0f);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);
  R* Ld = rp<R>(P.Ld);
  R* Lo = rp<R>(P.Lo);
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* GG = rp<R>(P.G);
  for (int i = 0; i <= N; ++i) {
    const size_t o = (size_t)i * kNN + l;
    Ld[o] = r_fma(beta, r_fma(two, GG[o], Kd[o]), cL * Ld[o]) * inv;
    if (i < N) Lo[o] = r_fma(beta, Ko[o], cL * Lo[o]) * inv;
  }
}

// One iteration of Alg. 1 for the plan of these sixteen lanes: quadrature
// (one state per lane), bisection over beta (App. C, the decisions of
// iterate_once), update.
template <typename QT, typename R>
PGV_BIG void iterate_lane(const Lane& x, const PlanDesc& P) {
  double* sc = P.scal;
  __syncwarp(x.mask);
  if (temp_switch_due(P)) {
    __syncwarp(x.mask);
    switch_temperature<kN, R>(P, x.l, 16);
    __syncwarp(x.mask);
  }
  const int cur = (int)sc[S_CUR];
  const int oa = (cur + 1) % 3, ob = (cur + 2) % 3;
  const int N = P.N;
  double coll = 0.0;
  bool qok = true;
  {
    const R* mu = rp<R>(P.mu[cur]);
    const R* Sd = rp<R>(P.Sd[cur]);
    R* gg = rp<R>(P.g);
    R* GGw = rp<R>(P.G);
    double part = 0.0;
    for (int i = x.l; i <= N; i += 16) {
      R mu_i[kN], S_ii[kNN], g[kN], G[kNN];
      double m0;
      ld_vec<kN, R>(mu + (size_t)i * kN, mu_i);
      ld_blk<kN, R>(Sd + (size_t)i * kNN, S_ii);
      qok = quad_factor<kN, QT, R>(P, i, mu_i, S_ii, g, G, m0) && qok;
      st_vec<kN, R>(gg + (size_t)i * kN, g);
      st_blk<kN, R>(GGw + (size_t)i * kNN, G);
      part += m0;
    }
    coll = halfsum_d(x, part);
    qok = __all_sync(x.mask, qok);
  }
  __syncwarp(x.mask);
  if (!qok) {
    if (x.l == 0) sc[S_STATUS] = 3.0;
    __syncwarp(x.mask);
    return;
  }
  const double logdet_k = sc[S_LOGDET];
  const double prior_k = sc[S_PRIOR];
  const int k = (int)sc[S_K];
  const double eps = P.kl_eps;
  const bool has_eps = isfinite(eps) && eps > 0.0;
  double margin = INFINITY;
  int trials = 0, best = -1;
  TrialOut bestR;
  double best_beta = 0.0;
  bestR.kl = 0.0;
  bestR.logdet = logdet_k;
  bestR.prior_cost = prior_k;
  double beta = P.beta_max, lo = 0.0, hi = P.beta_max;
  int into = oa, halvings = 0;
  bool searching = false;
  for (;;) {
    TrialOut Rt = trial_lane<R>(x, P, beta, cur, into, logdet_k);
    __syncwarp(x.mask);
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
  if (best >= 0) accept_lane<R>(x, P, best_beta);
  __syncwarp(x.mask);
  if (x.l == 0) {
    if (k < P.log_cap) {
      pgvimp_step_info li;
      li.beta = best_beta;
      li.kl = (best >= 0) ? bestR.kl : 0.0;
      li.kl_margin = margin;
      li.prior_cost = prior_k;
      li.collision_cost = coll;
      li.entropy = 0.5 * ((double)P.n * (P.N + 1) * ln_2pie() - logdet_k);
      li.trials = trials;
      li.iter = k;
      P.log[k] = li;
    }
    if (best >= 0) {
      sc[S_CUR] = (double)best;
      sc[S_LOGDET] = bestR.logdet;
      sc[S_PRIOR] = bestR.prior_cost;
    }
    sc[S_COLL] = coll;
    sc[S_K] = (double)(k + 1);
    sc[S_KIN] = sc[S_KIN] + 1.0;
  }
  __syncwarp(x.mask);
}

}  // namespace lanef

// Fused iterations in the lane form: blockDim.x / 16 plans per block.
// Resident blocks of 128 threads per SM the register allocation targets.
// Eight blocks of 128 threads per SM (64 registers a thread) measured fastest:
// 18,944 dense-horizon plans x 30 iterations with double-float recursions in
// 5.08 s on B300, against 5.14 s at six blocks; with the compiler's own
// register count (168, three blocks) an earlier build was 26% slower.
#ifndef PGV_LANE_MIN_BLOCKS
#define PGV_LANE_MIN_BLOCKS 8
#endif
template <typename QT, typename R>
__global__ void __launch_bounds__(128, PGV_LANE_MIN_BLOCKS) k_iterate_lane(const PlanDesc* __restrict__ descs,
                                                                           int count, int iters) {
  const int p = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 4);
  if (p >= count) return;
  const lanef::Lane x = lanef::make_lane();
  const PlanDesc& P = descs[p];
  for (int it = 0; it < iters; ++it) {
    if (P.scal[S_STATUS] != 0.0 || P.scal[S_INIT] == 0.0) return;
    if ((int)P.scal[S_KIN] >= P.iters) return;
    lanef::iterate_lane<QT, R>(x, P);
  }
}

template <typename QT, typename R>
cudaError_t launch_iter_lane(const Launch& L, int iters) {
  const int tpb = 128;
  const long threads = (long)L.count * 16;
  k_iterate_lane<QT, R><<<(unsigned)((threads + tpb - 1) / tpb), tpb, 0, L.stream>>>(L.descs, L.count, iters);
  return cudaGetLastError();
}

}  // namespace pgv
