// pgvimp_cr.cuh -- the latency form of the fused iteration: one thread block
// per plan, the time axis spread over the block's threads.
//
// The block recursions of the hot path (marginals, Sec. 5.1; the Thm 1 solve,
// log det and selected inverse) are chains over N+1 states.  Here they run
// by block cyclic reduction: at level h = 1, 2, 4, ... the states that are odd
// multiples of h are eliminated in parallel (their neighbours at distance h
// receive Schur-complement updates and a new coupling at distance 2h), and the
// backward pass recovers, level by level in reverse, the mean correction and
// the selected blocks Sigma_ii, Sigma_{i+1,i}.  This is Cholesky of the same
// SPD matrix under another elimination order (numerically as stable as the
// sequential sweep), with depth 2 log2(N) instead of 2N; it does about twice
// the sequential flops, which is what a latency form spends.
//
// Per state, an eliminated block i with neighbours l = i - h, r = i + h keeps
//   D_i^-1 (packed), U_l = D_i^-1 A_{i,l}, U_r = D_i^-1 A_{i,r}
// and the backward pass evaluates
//   Sigma_{i,l} = -(U_l Sigma_ll + U_r Sigma_rl),
//   Sigma_{i,r} = -(U_l Sigma_lr + U_r Sigma_rr),
//   Sigma_ii    = D_i^-1 - Sigma_{i,l} U_l^T - Sigma_{i,r} U_r^T,
//   x_i         = y_i - U_l x_l - U_r x_r,   y_i = D_i^-1 (reduced rhs)_i.
// Sigma_rl is the cross block of l and r, which are neighbours one level up;
// cross blocks live in slot min(l, r) of the So buffer, so that after level 1
// slot j holds Sigma_{j+1,j}.
#pragma once
#include "pgvimp_crw.cuh"
#include "pgvimp_kernels.cuh"

namespace pgv {

// The warp-cooperative form of the trial (pgvimp_crw.cuh) serves n >= 6, whose
// blocks do not fit one thread's registers; n = 4 keeps one thread per
// elimination.
template <int n>
constexpr bool kCrWarp = (n >= 6);

// Per-state scratch of the cyclic reduction (R elements, 16-byte aligned
// sub-blocks): working diagonal blocks of both systems (their inverses after
// elimination), couplings, the four U blocks, the reduced rhs and the mean
// correction.
template <int n>
struct CrScr {
  static constexpr int nn = n * n, np = n * (n + 1) / 2, npe = np + (np & 1);
  static constexpr int oDA = 0, oDM = npe, oCA = 2 * npe, oCM = oCA + nn, oUlA = oCM + nn, oUrA = oUlA + nn,
                       oUlM = oUrA + nn, oUrM = oUlM + nn, oR = oUrM + nn, oX = oR + n;
  static constexpr int stride = oX + n;
};

// ------------------------------------------------------------ block helpers

// Z = S X^T, S symmetric packed.
template <int n, typename R>
PGV_DEV void mul_sym_fullT(const R* S, const R* X, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) {
      R s = S[pk(a, 0)] * X[c * n];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 1; t < n; ++t) s = r_fma(S[pk(a, t)], X[c * n + t], s);
      Z[a * n + c] = s;
    }
}
// packed Z -= X Y (product known symmetric)
template <int n, typename R>
PGV_DEV void sub_nn_packed(R* Z, const R* X, const R* Y) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = Z[pk(a, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 0; t < n; ++t) s = r_fma(-X[a * n + t], Y[t * n + c], s);
      Z[pk(a, c)] = s;
    }
}
// packed Z -= X^T Y (product known symmetric)
template <int n, typename R>
PGV_DEV void sub_tn_packed(R* Z, const R* X, const R* Y) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = Z[pk(a, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 0; t < n; ++t) s = r_fma(-X[t * n + a], Y[t * n + c], s);
      Z[pk(a, c)] = s;
    }
}
// Z = -(X Y), or Z -= X Y with `accumulate`; full n x n.
template <int n, typename R>
PGV_DEV void mul_nn_sub(const R* X, const R* Y, R* Z, bool accumulate) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) {
      R s = accumulate ? Z[a * n + c] : r_fromf<R>(0.0f);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 0; t < n; ++t) s = r_fma(-X[a * n + t], Y[t * n + c], s);
      Z[a * n + c] = s;
    }
}
// packed Z = Dinv - X U^T - Y V^T  (symmetric result); Y/V may be null.
template <int n, typename R>
PGV_DEV void schur_back_packed(const R* Dinv, const R* X, const R* U, const R* Y, const R* V, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = Dinv[pk(a, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 0; t < n; ++t) s = r_fma(-X[a * n + t], U[c * n + t], s);
      if (Y) {
#pragma unroll (n <= 8 ? 32 : 0)
        for (int t = 0; t < n; ++t) s = r_fma(-Y[a * n + t], V[c * n + t], s);
      }
      Z[pk(a, c)] = s;
    }
}
// y = S v (S symmetric packed)
template <int n, typename R>
PGV_DEV void sym_mv(const R* S, const R* v, R* y) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a) {
    R s = S[pk(a, 0)] * v[0];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 1; c < n; ++c) s = r_fma(S[pk(a, c)], v[c], s);
    y[a] = s;
  }
}
// y -= X v (trans = false) or y -= X^T v (trans = true)
template <int n, typename R>
PGV_DEV void sub_mv(const R* X, const R* v, R* y, bool trans) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a) {
    R s = y[a];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) s = r_fma(-(trans ? X[c * n + a] : X[a * n + c]), v[c], s);
    y[a] = s;
  }
}

// The root's pivot block inverse, out of line.  (Inlined, the double-float
// n = 4 build miscomputed the root pivot at the default front-end
// optimisation; a stand-alone reduction built from these headers is exact
// with this call out of line, or inlined at -O1, -O0 or with -G.)
template <int n, typename R>
__device__ __noinline__ void root_chol_inverse(const R* C, R* Cinv, LogDetAcc<R>& ld, bool& ok) {
  chol_inverse<n, R>(C, Cinv, ld, ok);
}

// ------------------------------------------------------------ trial (a5), cyclic reduction

// Thm 1 at step beta, in the scaled form of `trial` (A~ = beta (2G + K^-1) +
// Lambda_k = (beta+1) Lambda', M = beta K^-1 + Lambda_k, M delta = beta (b - g
// - K^-1 mu_k)), by cyclic reduction over the thread block.  With
// `marg_only` it computes the marginals of Lambda_k alone (A~ = Lambda_k, no
// mean system) into set `out` with the prior cost of mu[cur].  Every thread
// returns the same TrialOut.
template <int n, typename R>
PGV_BIG TrialOut cr_trial(const PlanDesc& P, double beta_d, int cur, int out, double logdet_k, bool marg_only,
                          double* red) {
  using S = CrScr<n>;
  constexpr int nn = n * n, np = S::np, SS = S::stride;
  const int N = P.N, tid = threadIdx.x, T = blockDim.x;
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
  R* mo_out = rp<R>(P.mu[out]);
  R* Sd_out = rp<R>(P.Sd[out]);
  R* So_out = rp<R>(P.So[out]);
  const bool wm = !marg_only;
  const R beta = r_from<R>(beta_d), beta2 = beta + beta, zero = r_fromf<R>(0.0f);
  // natural-gradient step (Sec. 3.1(d)): Lambda_k weighted by 1 - beta, M = A~, s = 1
  const bool ngd = wm && (P.update == PGVIMP_UPDATE_NGD);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);
  TrialOut res;
  res.kl = INFINITY;
  res.pd = false;
  res.logdet = 0.0;
  res.prior_cost = 0.0;
  res.delta = 0.0;
  res.trace = 0.0;

  // ---- level-0 system: diagonal blocks, couplings, right-hand side
  for (int i = tid; i <= N; i += T) {
    R* sp = scr + (size_t)i * SS;
    R B[nn], DA[np], DM[np];
    ld_blk<n, R>(Ld + (size_t)i * nn, B);
    if (ngd)
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < nn; ++e) B[e] = cL * B[e];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
      for (int c = 0; c <= a; ++c) DA[pk(a, c)] = DM[pk(a, c)] = B[a * n + c];
    if (wm) {
      R K[nn], G[nn];
      ld_blk<n, R>(Kd + (size_t)i * nn, K);
      ld_blk<n, R>(GG + (size_t)i * nn, G);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c <= a; ++c) {
          const R kb = beta * K[a * n + c];
          DM[pk(a, c)] = DM[pk(a, c)] + kb;
          if (ngd) DM[pk(a, c)] = r_fma(beta2, G[a * n + c], DM[pk(a, c)]);
          DA[pk(a, c)] = r_fma(beta2, G[a * n + c], DA[pk(a, c)] + kb);
        }
      // rhs_i = beta (b_i - g_i - (K^-1 mu)_i)
      R mi[n], Kmu[n];
      ld_vec<n, R>(mu + (size_t)i * n, mi);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) {
        R s = zero;
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) s = r_fma(K[a * n + c], mi[c], s);
        Kmu[a] = s;
      }
      if (i > 0) {
        R E[nn], mp[n];
        ld_blk<n, R>(Ko + (size_t)(i - 1) * nn, E);   // K^-1_{i,i-1}
        ld_vec<n, R>(mu + (size_t)(i - 1) * n, mp);
#pragma unroll (n <= 8 ? 32 : 0)
        for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
          for (int c = 0; c < n; ++c) Kmu[a] = r_fma(E[a * n + c], mp[c], Kmu[a]);
      }
      if (i < N) {
        R E[nn], mn[n];
        ld_blk<n, R>(Ko + (size_t)i * nn, E);         // K^-1_{i+1,i}; block (i, i+1) is its transpose
        ld_vec<n, R>(mu + (size_t)(i + 1) * n, mn);
#pragma unroll (n <= 8 ? 32 : 0)
        for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
          for (int c = 0; c < n; ++c) Kmu[a] = r_fma(E[c * n + a], mn[c], Kmu[a]);
      }
      R rhs[n];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) rhs[a] = beta * ((bb[(size_t)i * n + a] - gg[(size_t)i * n + a]) - Kmu[a]);
      st_vec<n, R>(sp + S::oR, rhs);
      st_packed<n, R>(sp + S::oDM, DM);
    }
    st_packed<n, R>(sp + S::oDA, DA);
    if (i < N) {
      R E[nn];
      ld_blk<n, R>(Lo + (size_t)i * nn, E);
      if (ngd)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int e = 0; e < nn; ++e) E[e] = cL * E[e];
      if (wm) {
        R K[nn];
        ld_blk<n, R>(Ko + (size_t)i * nn, K);
#pragma unroll (n <= 8 ? 32 : 0)
        for (int e = 0; e < nn; ++e) E[e] = r_fma(beta, K[e], E[e]);   // beta K^-1_{i+1,i} + Lambda_{i+1,i}
        st_blk<n, R>(sp + S::oCM, E);
      }
      st_blk<n, R>(sp + S::oCA, E);
    }
  }
  __syncthreads();

  // ---- forward: eliminate the odd multiples of h
  LogDetAcc<R> ldA, ldM;
  ldA.init();
  ldM.init();
  bool okA = true, okM = true;
  int h = 1;
  for (; h <= N; h <<= 1) {
    for (int i = h + 2 * h * tid; i <= N; i += 2 * h * T) {
      R* sp = scr + (size_t)i * SS;
      const R* spl = scr + (size_t)(i - h) * SS;
      const bool hasr = (i + h <= N);
      {
        R D[np], Di[np], C[nn], U[nn];
        ld_packed<n, R>(sp + S::oDA, D);
        chol_inverse<n, R>(D, Di, ldA, okA);
        st_packed<n, R>(sp + S::oDA, Di);
        ld_blk<n, R>(spl + S::oCA, C);                // A_{i,l}
        mul_sym_full<n, R>(Di, C, U);
        st_blk<n, R>(sp + S::oUlA, U);
        if (hasr) {
          ld_blk<n, R>(sp + S::oCA, C);               // A_{r,i}; A_{i,r} = its transpose
          mul_sym_fullT<n, R>(Di, C, U);
          st_blk<n, R>(sp + S::oUrA, U);
        }
      }
      if (wm) {
        R D[np], Di[np], C[nn], U[nn], v[n], y[n];
        ld_packed<n, R>(sp + S::oDM, D);
        chol_inverse<n, R>(D, Di, ldM, okM);
        st_packed<n, R>(sp + S::oDM, Di);
        ld_blk<n, R>(spl + S::oCM, C);
        mul_sym_full<n, R>(Di, C, U);
        st_blk<n, R>(sp + S::oUlM, U);
        if (hasr) {
          ld_blk<n, R>(sp + S::oCM, C);
          mul_sym_fullT<n, R>(Di, C, U);
          st_blk<n, R>(sp + S::oUrM, U);
        }
        ld_vec<n, R>(sp + S::oR, v);
        sym_mv<n, R>(Di, v, y);
        st_vec<n, R>(sp + S::oR, y);                  // y_i = D_i^-1 rhs_i
      }
    }
    __syncthreads();
    // survivors j (multiples of 2h): Schur updates from j - h and j + h
    for (int j = 2 * h * tid; j <= N; j += 2 * h * T) {
      R* sp = scr + (size_t)j * SS;
      const bool hasl = (j >= h), hasr = (j + h <= N), has2 = (j + 2 * h <= N);
      const R* spl = scr + (size_t)(hasl ? j - h : j) * SS;
      const R* spr = scr + (size_t)(hasr ? j + h : j) * SS;
      {
        R D[np], C[nn], U[nn];
        ld_packed<n, R>(sp + S::oDA, D);
        if (hasl) {
          ld_blk<n, R>(spl + S::oCA, C);              // A_{j,i}, i = j - h
          ld_blk<n, R>(spl + S::oUrA, U);
          sub_nn_packed<n, R>(D, C, U);
        }
        if (hasr) {
          R Cj[nn];
          ld_blk<n, R>(sp + S::oCA, Cj);              // A_{i,j}, i = j + h
          ld_blk<n, R>(spr + S::oUlA, U);
          sub_tn_packed<n, R>(D, Cj, U);
          if (has2) {
            ld_blk<n, R>(spr + S::oCA, C);            // A_{j+2h,i}
            mul_nn_sub<n, R>(C, U, Cj, false);        // A_{j+2h,j} = -A_{j+2h,i} U_l(i)
            st_blk<n, R>(sp + S::oCA, Cj);
          }
        }
        st_packed<n, R>(sp + S::oDA, D);
      }
      if (wm) {
        R D[np], C[nn], U[nn], r[n], y[n];
        ld_packed<n, R>(sp + S::oDM, D);
        ld_vec<n, R>(sp + S::oR, r);
        if (hasl) {
          ld_blk<n, R>(spl + S::oCM, C);
          ld_blk<n, R>(spl + S::oUrM, U);
          sub_nn_packed<n, R>(D, C, U);
          ld_vec<n, R>(spl + S::oR, y);
          sub_mv<n, R>(C, y, r, false);
        }
        if (hasr) {
          R Cj[nn];
          ld_blk<n, R>(sp + S::oCM, Cj);
          ld_blk<n, R>(spr + S::oUlM, U);
          sub_tn_packed<n, R>(D, Cj, U);
          ld_vec<n, R>(spr + S::oR, y);
          sub_mv<n, R>(Cj, y, r, true);
          if (has2) {
            ld_blk<n, R>(spr + S::oCM, C);
            mul_nn_sub<n, R>(C, U, Cj, false);
            st_blk<n, R>(sp + S::oCM, Cj);
          }
        }
        st_packed<n, R>(sp + S::oDM, D);
        st_vec<n, R>(sp + S::oR, r);
      }
    }
    __syncthreads();
  }
  // ---- root (state 0)
  if (tid == 0) {
    R* sp = scr;
    R D[np], Di[np];
    ld_packed<n, R>(sp + S::oDA, D);
    root_chol_inverse<n, R>(D, Di, ldA, okA);
    st_packed<n, R>(sp + S::oDA, Di);
    st_sym<n, R>(Sd_out, Di);
    if (wm) {
      R v[n], y[n];
      ld_packed<n, R>(sp + S::oDM, D);
      chol_inverse<n, R>(D, Di, ldM, okM);
      ld_vec<n, R>(sp + S::oR, v);
      sym_mv<n, R>(Di, v, y);
      st_vec<n, R>(sp + S::oX, y);
    }
  }
  const bool pd = __syncthreads_and(okA && okM);
  double lsum[1] = {ldA.log_value()};
  block_sum<1>(lsum, red);
  if (!pd) return res;

  // ---- backward: selected inverse and back substitution, top level first
  for (h >>= 1; h >= 1; h >>= 1) {
    for (int i = h + 2 * h * tid; i <= N; i += 2 * h * T) {
      const int l = i - h, r = i + h;
      const bool hasr = (r <= N);
      const R* sp = scr + (size_t)i * SS;
      {
        R Sll[np], Ul[nn], Sil[nn];
        ld_sym<n, R>(Sd_out + (size_t)l * nn, Sll);
        ld_blk<n, R>(sp + S::oUlA, Ul);
        mul_full_sym<n, R>(Ul, Sll, Sil);             // U_l Sigma_ll
        R Ur[nn], Sir[nn];
        if (hasr) {
          R Srl[nn], Srr[np];
          ld_blk<n, R>(So_out + (size_t)l * nn, Srl);   // Sigma_{r,l}
          ld_sym<n, R>(Sd_out + (size_t)r * nn, Srr);
          ld_blk<n, R>(sp + S::oUrA, Ur);
          mul_full_sym<n, R>(Ur, Srr, Sir);           // U_r Sigma_rr
#pragma unroll (n <= 8 ? 32 : 0)
          for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
            for (int c = 0; c < n; ++c) {
              R s = Sil[a * n + c], t = Sir[a * n + c];
#pragma unroll (n <= 8 ? 32 : 0)
              for (int k = 0; k < n; ++k) {
                s = r_fma(Ur[a * n + k], Srl[k * n + c], s);   // + U_r Sigma_rl
                t = r_fma(Ul[a * n + k], Srl[c * n + k], t);   // + U_l Sigma_lr
              }
              Sil[a * n + c] = -s;
              Sir[a * n + c] = -t;
            }
        } else {
#pragma unroll (n <= 8 ? 32 : 0)
          for (int e = 0; e < nn; ++e) Sil[e] = -Sil[e];
        }
        R Di[np], Sii[np];
        ld_packed<n, R>(sp + S::oDA, Di);
        schur_back_packed<n, R>(Di, Sil, Ul, hasr ? Sir : nullptr, hasr ? Ur : nullptr, Sii);
        st_sym<n, R>(Sd_out + (size_t)i * nn, Sii);
        st_blk<n, R>(So_out + (size_t)l * nn, Sil);   // Sigma_{i,l} = Sigma_{l+h,l}
        if (hasr) {
          R X[nn];
#pragma unroll (n <= 8 ? 32 : 0)
          for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
            for (int c = 0; c < n; ++c) X[a * n + c] = Sir[c * n + a];
          st_blk<n, R>(So_out + (size_t)i * nn, X);   // Sigma_{r,i}
        }
      }
      if (wm) {
        R x[n], v[n], U[nn];
        ld_vec<n, R>(sp + S::oR, x);
        ld_blk<n, R>(sp + S::oUlM, U);
        ld_vec<n, R>(scr + (size_t)l * SS + S::oX, v);
        sub_mv<n, R>(U, v, x, false);
        if (hasr) {
          ld_blk<n, R>(sp + S::oUrM, U);
          ld_vec<n, R>(scr + (size_t)r * SS + S::oX, v);
          sub_mv<n, R>(U, v, x, false);
        }
        st_vec<n, R>(scr + (size_t)i * SS + S::oX, x);
      }
    }
    __syncthreads();
  }

  // ---- KL pieces, prior cost, outputs scaled by s (beta + 1, or 1 for the natural-gradient step)
  const double bp1d = ngd ? 1.0 : beta_d + 1.0;
  const R bp1 = r_from<R>(bp1d);
  R trc = zero, dl = zero, ktr = zero, kq = zero;
  for (int i = tid; i <= N; i += T) {
    R Si[np], xi[n], dpi[n], mo[n];
    ld_sym<n, R>(Sd_out + (size_t)i * nn, Si);
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) xi[a] = zero;
    if (wm) ld_vec<n, R>(scr + (size_t)i * SS + S::oX, xi);
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a) {
      mo[a] = mu[(size_t)i * n + a] + xi[a];
      dpi[a] = mo[a] - mubar[(size_t)i * n + a];
    }
    R B[nn];
    if (wm) {
      ld_blk<n, R>(Ld + (size_t)i * nn, B);
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
    }
    ld_blk<n, R>(Kd + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
    for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
      for (int c = 0; c < n; ++c) {
        trc = r_fma(-B[a * n + c], Si[pk(a, c)], trc);
        ktr = r_fma(B[a * n + c], Si[pk(a, c)], ktr);
        kq = r_fma(dpi[a] * B[a * n + c], dpi[c], kq);
      }
    if (i < N) {
      R So[nn], xn[n], dpn[n];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) xn[a] = zero;
      if (wm) ld_vec<n, R>(scr + (size_t)(i + 1) * SS + S::oX, xn);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a) dpn[a] = (mu[(size_t)(i + 1) * n + a] + xn[a]) - mubar[(size_t)(i + 1) * n + a];
      ld_blk<n, R>(So_out + (size_t)i * nn, So);     // Sigma~_{i+1,i}
      if (wm) {
        ld_blk<n, R>(Lo + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
        for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
          for (int c = 0; c < n; ++c) {
            trc = r_fma(B[a * n + c] + B[a * n + c], So[a * n + c], trc);
            dl = r_fma((xn[a] + xn[a]) * B[a * n + c], xi[c], dl);
          }
      }
      ld_blk<n, R>(Ko + (size_t)i * nn, B);
#pragma unroll (n <= 8 ? 32 : 0)
      for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
        for (int c = 0; c < n; ++c) {
          trc = r_fma(-(B[a * n + c] + B[a * n + c]), So[a * n + c], trc);
          ktr = r_fma(B[a * n + c] + B[a * n + c], So[a * n + c], ktr);
          kq = r_fma((dpn[a] + dpn[a]) * B[a * n + c], dpi[c], kq);
        }
      if (wm) {
#pragma unroll (n <= 8 ? 32 : 0)
        for (int e = 0; e < nn; ++e) So[e] = bp1 * So[e];
        st_blk<n, R>(So_out + (size_t)i * nn, So);
      }
    }
    if (wm) {
#pragma unroll (n <= 8 ? 32 : 0)
      for (int e = 0; e < np; ++e) Si[e] = bp1 * Si[e];
      st_sym<n, R>(Sd_out + (size_t)i * nn, Si);
      st_vec<n, R>(mo_out + (size_t)i * n, mo);
    }
  }
  double parts[4] = {r_to(trc), r_to(dl), r_to(ktr), r_to(kq)};
  block_sum<4>(parts, red);
  res.pd = true;
  const double Dd = (double)n * (N + 1);
  res.logdet = lsum[0] - ((wm && !ngd) ? Dd * log(bp1d) : 0.0);
  res.trace = beta_d * parts[0];
  res.delta = parts[1];
  res.kl = 0.5 * (res.trace + res.delta + res.logdet - logdet_k);
  res.prior_cost = 0.5 * (bp1d * parts[2] + parts[3]);
  return res;
}

// ------------------------------------------------------------ iteration (Alg. 1 loop body), block form

template <int n, typename R>
PGV_BIG void cr_accept_precision(const PlanDesc& P, double beta_d) {
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
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
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

// Same decisions as iterate_once (App. C bisection, feasibility in FP64),
// with the quadrature spread over the block's threads and cyclic-reduction
// trials.
template <int n, typename QT, typename R>
PGV_BIG void cr_iterate_once(const PlanDesc& P, double* red, R* wsm) {
  constexpr int nn = n * n;
  double* sc = P.scal;
  if (temp_switch_due(P)) {            // uniform: every thread reads the same slots
    __syncthreads();
    switch_temperature<n, R>(P, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  const int cur = (int)sc[S_CUR];
  const int oa = (cur + 1) % 3, ob = (cur + 2) % 3;
  const int N = P.N;
  double coll;
  {
    const R* mu = rp<R>(P.mu[cur]);
    const R* Sd = rp<R>(P.Sd[cur]);
    R* gg = rp<R>(P.g);
    R* GG = rp<R>(P.G);
    bool ok = true;
    double part[1] = {0.0};
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
      R mu_i[n], S_ii[nn], g[n], G[nn];
      double m0;
      ld_vec<n, R>(mu + (size_t)i * n, mu_i);
      ld_blk<n, R>(Sd + (size_t)i * nn, S_ii);
      ok = quad_factor<n, QT, R>(P, i, mu_i, S_ii, g, G, m0) && ok;
      st_vec<n, R>(gg + (size_t)i * n, g);
      st_blk<n, R>(GG + (size_t)i * nn, G);
      part[0] += m0;
    }
    ok = __syncthreads_and(ok);
    block_sum<1>(part, red);
    coll = part[0];
    if (!ok) {
      __syncthreads();
      if (threadIdx.x == 0) sc[S_STATUS] = 3.0;
      __syncthreads();
      return;
    }
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
    TrialOut Rt;
    if constexpr (kCrWarp<n>) Rt = crw::trial<n, R>(P, beta, cur, into, logdet_k, false, red, wsm);
    else Rt = cr_trial<n, R>(P, beta, cur, into, logdet_k, false, red);
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
  if (best >= 0) {
    if constexpr (kCrWarp<n>) crw::accept_precision<n, R>(P, best_beta);
    else cr_accept_precision<n, R>(P, best_beta);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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
  __syncthreads();
}

// Initial iterate (as init_plan) with its marginals by cyclic reduction.
template <int n, typename R>
PGV_BIG void cr_init_plan(const PlanDesc& P, double* red, R* wsm) {
  constexpr int nn = n * n;
  double* sc = P.scal;
  const int N = P.N, nq = P.nq;
  R* mu0 = rp<R>(P.mu[0]);
  R* Ld = rp<R>(P.Ld);
  R* Lo = rp<R>(P.Lo);
  const R zero = r_fromf<R>(0.0f), sI = r_from<R>(P.init_scale);
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    double s = (double)i / N;
    for (int a = 0; a < nq; ++a) {
      double d = P.muN[a] - P.mu0[a];
      mu0[(size_t)i * n + a] = r_from<R>(P.mu0[a] + s * d);
      mu0[(size_t)i * n + nq + a] = r_from<R>(d / P.T);
    }
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
  __syncthreads();
  TrialOut M;
  if constexpr (kCrWarp<n>) M = crw::trial<n, R>(P, 0.0, 0, 0, 0.0, true, red, wsm);
  else M = cr_trial<n, R>(P, 0.0, 0, 0, 0.0, true, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!M.pd) {
      sc[S_STATUS] = 2.0;
    } else {
      sc[S_CUR] = 0.0;
      sc[S_LOGDET] = M.logdet;
      sc[S_PRIOR] = M.prior_cost;
      sc[S_K] = 0.0;
      sc[S_KIN] = 0.0;
      sc[S_INIT] = 1.0;
      sc[S_FMT] = 0.0;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ kernels (one block per plan)

// Dynamic shared memory of a block-form launch: the per-warp staging of the
// warp-cooperative trial, none otherwise.
template <int n, typename R>
constexpr size_t cr_dyn_smem(int tpb) {
  return kCrWarp<n> ? (size_t)(tpb / 32) * crw::Lay<n>::ws * sizeof(R) : 0;
}

template <int n, typename QT, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_iterate_cta(const PlanDesc* __restrict__ descs, int count,
                                                               int iters) {
  __shared__ double red[(kCrMaxThreads / 32) * 4];
  extern __shared__ __align__(16) unsigned char cr_dyn[];
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  for (int it = 0; it < iters; ++it) {
    if (P.scal[S_STATUS] != 0.0 || P.scal[S_INIT] == 0.0) return;
    if ((int)P.scal[S_KIN] >= P.iters) return;
    cr_iterate_once<n, QT, R>(P, red, reinterpret_cast<R*>(cr_dyn));
  }
}

template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_init_cta(const PlanDesc* __restrict__ descs, int count) {
  __shared__ double red[(kCrMaxThreads / 32) * 4];
  extern __shared__ __align__(16) unsigned char cr_dyn[];
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  if (P.scal[S_STATUS] != 0.0) return;
  cr_init_plan<n, R>(P, red, reinterpret_cast<R*>(cr_dyn));
}

// ------------------------------------------------------------ SLR and the LTV prior (a6, a0), block form

// SLR linearisation (Sec. 6.2) with the states spread over the block; modes as
// k_slr (1: straight-line nominal with K0; 0: current iterate, closing the
// previous outer iteration's norm; 2: current iterate without bookkeeping).
template <int n, typename QT, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_slr_cta(const PlanDesc* __restrict__ descs, int count, int mode) {
  constexpr int nn = n * n;
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  if (P.scal[S_STATUS] != 0.0) return;
  if (mode == 0 && threadIdx.x == 0) {
    const int j = (int)P.scal[S_J];
    if (j < P.slr_iters) P.slr_norms[j] = slr_norm<n, R>(P);   // reads the previous nominal
    P.scal[S_J] = (double)(j + 1);
  }
  __syncthreads();
  const int N = P.N, nq = P.nq;
  const bool first = (mode == 1);
  const int cur = (int)P.scal[S_CUR];
  const R* mu = rp<R>(P.mu[cur]);
  const R* Sd = rp<R>(P.Sd[cur]);
  bool ok = true;
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    double xb[n], Sb[nn];
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
  ok = __syncthreads_and(ok);
  if (!ok && threadIdx.x == 0) P.scal[S_STATUS] = 4.0;
}

// The GP prior (Sec. 3; the prior step of Alg. 1; for mode 1 the SLR linearisation's
// LTV prior of Alg. 2) with its work spread over the block.  First the Van
// Loan factors Phi_i, Q_i, u_i, one thread per step (a single step for a
// time-invariant system), stored to the per-step scratch with scalar stores.
// Then one warp per state assembles, in shared memory with the warp
// routines of pgvimp_crw.cuh (FP64),
//   K^-1_ii = C_i + Phi_i^T Q_i^-1 Phi_i,   b_i = c_i - Phi_i^T Q_i^-1 u_i,
//   K^-1_{i+1,i} = -Q_i^-1 Phi_i,
// with the carries C_0 = K_0^-1, c_0 = K_0^-1 mu_0, C_i = Q_{i-1}^-1,
// c_i = Q_{i-1}^-1 u_{i-1}, and at i = N the terminal K_N^-1, K_N^-1 mu_N in
// place of the step terms (the expressions of prior_build), all scaled by the
// current inverse temperature.  mu_bar follows in k_prior_solve_cta.  (Built
// with thread-local n x n arrays on sm_103a, this assembly returned wrong
// blocks for some horizons and block widths; the warp form holds no block in
// thread-local memory.)
template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_prior_cta(const PlanDesc* __restrict__ descs, int count,
                                                             int mode) {
  constexpr int nn = n * n, SS = 2 * nn + n;
  using Ly = crw::Lay<n>;
  static_assert(sizeof(R) == sizeof(double), "the warp staging is sized in 8-byte elements");
  extern __shared__ __align__(16) unsigned char cr_dyn[];
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  if (P.scal[S_STATUS] != 0.0) return;
  const bool use_ltv = (mode == 1);
  const bool lti = !use_ltv && !P.A_per_step && !P.a_per_step;
  const int N = P.N, m = P.m;
  double* scr = P.scr;
  bool ok = true;
  {
    const int steps = lti ? 1 : N;
    for (int i = threadIdx.x; i < steps; i += blockDim.x) {
      double Wn[nn], A[nn], av[n], Phi[nn], Q[nn], u[n];
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double s = 0.0;
          for (int k = 0; k < m; ++k)
            for (int l = 0; l < m; ++l) s += P.B[r * m + k] * P.Qc[k * m + l] * P.B[c * m + l];
          Wn[r * n + c] = s;
        }
      const double* Ai = use_ltv ? P.Altv + (size_t)i * nn : (P.A_per_step ? P.A + (size_t)i * nn : P.A);
      for (int e = 0; e < nn; ++e) A[e] = Ai[e];
      for (int a = 0; a < n; ++a)
        av[a] = use_ltv ? P.altv[(size_t)i * n + a] : (P.a ? (P.a_per_step ? P.a[(size_t)i * n + a] : P.a[a]) : 0.0);
      ok = van_loan<n>(A, av, Wn, P.dt, Phi, Q, u) && ok;
      volatile double* sp = scr + (size_t)i * SS;
      for (int e = 0; e < nn; ++e) {
        sp[e] = Phi[e];
        sp[nn + e] = Q[e];
      }
      for (int a = 0; a < n; ++a) sp[2 * nn + a] = u[a];
    }
  }
  ok = __syncthreads_and(ok);
  const double it = cur_inv_temp(P);
  R* Kd = rp<R>(P.Kd);
  R* Ko = rp<R>(P.Ko);
  R* b = rp<R>(P.b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  double* ws = reinterpret_cast<double*>(cr_dyn) + (size_t)warp * Ly::ws;
  double* S0 = ws;            // carry C_i
  double* S1 = ws + nn;       // Phi_i, or K_N^-1
  double* S2 = ws + 2 * nn;   // Q_i^-1
  double* S3 = ws + 3 * nn;   // Phi_i^T Q_i^-1
  double* S4 = ws + 4 * nn;   // C_i + Phi^T Q^-1 Phi
  double* S5 = ws + 5 * nn;   // -Q_i^-1 Phi_i
  double* row = ws + Ly::oRow;
  double* col = ws + Ly::oCol;
  double* V0 = ws + Ly::oV;   // carry c_i
  double* V1 = V0 + n;        // u_{i-1}, mu_0; then u_i or mu_N
  double* V2 = V1 + n;        // b_i before scaling
  LogDetAcc<double> ldd;
  ldd.init();
  for (int i = warp; i <= N; i += NW) {
    // carry: K_0^-1 (c = K_0^-1 mu_0), or Q_{i-1}^-1 (c = Q_{i-1}^-1 u_{i-1})
    const double* spp = scr + (size_t)(lti ? 0 : (i > 0 ? i - 1 : 0)) * SS;
#pragma unroll 1
    for (int e = lane; e < nn; e += 32) S0[e] = (i == 0) ? P.K0[e] : spp[nn + e];
    if (lane < n) V1[lane] = (i == 0) ? P.mu0[lane] : spp[2 * nn + lane];
    crw::winv<n, double>(lane, S0, row, col, ldd, ok);
    crw::mv<n, double>(lane, S0, false, V1, nullptr, V0, false);
    __syncwarp();
    if (i < N) {
      const double* sp = scr + (size_t)(lti ? 0 : i) * SS;
#pragma unroll 1
      for (int e = lane; e < nn; e += 32) {
        S1[e] = sp[e];
        S2[e] = sp[nn + e];
      }
      if (lane < n) V1[lane] = sp[2 * nn + lane];
      crw::winv<n, double>(lane, S2, row, col, ldd, ok);
      crw::mm<n, double>(lane, S1, S2, nullptr, S3, 1, 0, 0);     // Phi^T Q^-1
      crw::mm<n, double>(lane, S2, S1, nullptr, S5, 0, 0, 1);     // -Q^-1 Phi
      __syncwarp();
      crw::mm<n, double>(lane, S3, S1, S0, S4, 0, 0, 0);          // C + Phi^T Q^-1 Phi
      crw::mv<n, double>(lane, S3, false, V1, V0, V2, true);      // c - Phi^T Q^-1 u
#pragma unroll 1
      for (int e = lane; e < nn; e += 32) Ko[(size_t)i * nn + e] = r_from<R>(S5[e] * it);
    } else {
#pragma unroll 1
      for (int e = lane; e < nn; e += 32) S1[e] = P.KN[e];
      if (lane < n) V1[lane] = P.muN[lane];
      crw::winv<n, double>(lane, S1, row, col, ldd, ok);
#pragma unroll 1
      for (int e = lane; e < nn; e += 32) S4[e] = S0[e] + S1[e];
      crw::mv<n, double>(lane, S1, false, V1, V0, V2, false);     // c + K_N^-1 mu_N
    }
    __syncwarp();
#pragma unroll 1
    for (int e = lane; e < nn; e += 32) {
      const int a = e / n, c = e - a * n;
      Kd[(size_t)i * nn + e] = r_from<R>((a == c ? S4[e] : 0.5 * (S4[e] + S4[c * n + a])) * it);
    }
    if (lane < n) b[(size_t)i * n + lane] = r_from<R>(V2[lane] * it);
    __syncwarp();
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) {
    P.scal[S_THIGH] = (P.inv_temp_high > 0.0 && it == P.inv_temp_high) ? 1.0 : 0.0;
    if (!ok) P.scal[S_STATUS] = 1.0;
  }
}

// mu_bar = K b (the prior mean) for the K^-1 and b just assembled, by the
// warp-cooperative block solve; a non-positive pivot marks the prior failed.
template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_prior_solve_cta(const PlanDesc* __restrict__ descs, int count) {
  extern __shared__ __align__(16) unsigned char cr_dyn[];
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  if (P.scal[S_STATUS] != 0.0) return;
  const bool ok = crw::solve<n, R>(P, rp<R>(P.Kd), rp<R>(P.Ko), rp<R>(P.b), rp<R>(P.mubar),
                                   reinterpret_cast<R*>(cr_dyn));
  if (!ok && threadIdx.x == 0) P.scal[S_STATUS] = 1.0;
}

// After a relinearisation (block form of k_relinearised): the prior cost
// 1/2 [tr(K^-1 Sigma) + (mu - mu_bar)^T K^-1 (mu - mu_bar)] of the current
// iterate under the new prior, summed over the block, and a fresh
// inner-iteration counter.
template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_relinearised_cta(const PlanDesc* __restrict__ descs, int count) {
  constexpr int nn = n * n;
  __shared__ double red[(kCrMaxThreads / 32) * 4];
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  if (P.scal[S_STATUS] != 0.0) return;
  const int N = P.N, s = (int)P.scal[S_CUR];
  const R* Kd = rp<R>(P.Kd);
  const R* Ko = rp<R>(P.Ko);
  const R* mu = rp<R>(P.mu[s]);
  const R* mubar = rp<R>(P.mubar);
  const R* Sd = rp<R>(P.Sd[s]);
  const R* So = rp<R>(P.So[s]);
  R tr = r_fromf<R>(0.0f), qd = r_fromf<R>(0.0f);
  for (int i = threadIdx.x; i <= N; i += blockDim.x) {
    R di[n], dn[n];
    for (int a = 0; a < n; ++a) di[a] = mu[(size_t)i * n + a] - mubar[(size_t)i * n + a];
    for (int e = 0; e < nn; ++e) tr = r_fma(Kd[(size_t)i * nn + e], Sd[(size_t)i * nn + e], tr);
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) qd = r_fma(di[a] * Kd[(size_t)i * nn + a * n + c], di[c], qd);
    if (i < N) {
      for (int a = 0; a < n; ++a) dn[a] = mu[(size_t)(i + 1) * n + a] - mubar[(size_t)(i + 1) * n + a];
      for (int e = 0; e < nn; ++e) {
        const R E = Ko[(size_t)i * nn + e];
        tr = r_fma(E + E, So[(size_t)i * nn + e], tr);
      }
      for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) qd = r_fma((dn[a] + dn[a]) * Ko[(size_t)i * nn + a * n + c], di[c], qd);
    }
  }
  double part[1] = {r_to(tr + qd)};
  block_sum<1>(part, red);
  if (threadIdx.x == 0) {
    P.scal[S_PRIOR] = 0.5 * part[0];
    P.scal[S_KIN] = 0.0;
  }
}

// Results in buffer set 0 and in FP64 (block form of k_finalize), element-
// parallel: the copy of the current set into set 0, then for double-float
// the in-place conversion of each element to double (the same thread owns
// element e in both loops).
template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_finalize_cta(const PlanDesc* __restrict__ descs, int count) {
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  const int cur = (int)P.scal[S_CUR];
  const bool fmt0 = (P.scal[S_FMT] == 0.0);
  const size_t N = P.N;
  const size_t cnt[5] = {(N + 1) * n, (N + 1) * n * n, N * n * n, (N + 1) * n * n, N * n * n};
  __syncthreads();   // every thread has read the flags before thread 0 rewrites them
  if (cur != 0 && fmt0) {
    R* dst[3] = {rp<R>(P.mu[0]), rp<R>(P.Sd[0]), rp<R>(P.So[0])};
    const R* src[3] = {rp<R>(P.mu[cur]), rp<R>(P.Sd[cur]), rp<R>(P.So[cur])};
    for (int k = 0; k < 3; ++k)
      for (size_t e = threadIdx.x; e < cnt[k]; e += blockDim.x) dst[k][e] = src[k][e];
  }
  if (!std::is_same<R, double>::value && fmt0) {
    double* bufs[5] = {P.mu[0], P.Sd[0], P.So[0], P.Ld, P.Lo};
    for (int k = 0; k < 5; ++k) {
      R* rbuf = rp<R>(bufs[k]);
      for (size_t e = threadIdx.x; e < cnt[k]; e += blockDim.x) {
        const double v = r_to(rbuf[e]);
        bufs[k][e] = v;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (cur != 0 && fmt0) P.scal[S_CUR] = 0.0;
    if (!std::is_same<R, double>::value && fmt0) P.scal[S_FMT] = 1.0;
  }
}

// Back to the working format (block form of k_working): double-float
// results converted in place from FP64, element-parallel.
template <int n, typename R>
__global__ void __launch_bounds__(kCrMaxThreads) k_working_cta(const PlanDesc* __restrict__ descs, int count) {
  if ((int)blockIdx.x >= count) return;
  const PlanDesc& P = descs[blockIdx.x];
  const bool fmt1 = (P.scal[S_FMT] == 1.0);
  __syncthreads();
  if (!std::is_same<R, double>::value && fmt1) {
    const size_t N = P.N;
    double* bufs[5] = {P.mu[0], P.Sd[0], P.So[0], P.Ld, P.Lo};
    const size_t cnt[5] = {(N + 1) * n, (N + 1) * n * n, N * n * n, (N + 1) * n * n, N * n * n};
    for (int k = 0; k < 5; ++k) {
      R* rbuf = rp<R>(bufs[k]);
      for (size_t e = threadIdx.x; e < cnt[k]; e += blockDim.x) {
        const R v = r_from<R>(bufs[k][e]);
        rbuf[e] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) P.scal[S_FMT] = 0.0;
  }
}

// Block form of the launch groups: `tpb` threads per plan (a multiple of 32,
// at most kCrMaxThreads).
template <int n, typename QT, typename R>
cudaError_t launch_iter_cta(const Launch& L, int iters, int tpb) {
  if (tpb < 32 || tpb > kCrMaxThreads || (tpb & 31)) return cudaErrorInvalidValue;
  const size_t smem = cr_dyn_smem<n, R>(tpb);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_iterate_cta<n, QT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_iterate_cta<n, QT, R><<<L.count, tpb, smem, L.stream>>>(L.descs, L.count, iters);
  return cudaGetLastError();
}

// The prior (`arg_i` = its mode), initial iterate, SLR linearisation
// (`arg_i` = mode), post-relinearisation prior cost, finalisation and return
// to the working format, block form, recursions in R (FP64 or double-float).
template <int n, typename R>
cudaError_t launch_aux_cta(const Launch& L, int phase, int arg_i, int qt32, int tpb) {
  if (tpb < 32 || tpb > kCrMaxThreads || (tpb & 31)) return cudaErrorInvalidValue;
  switch (phase) {
    case PH_INIT: {
      const size_t smem = cr_dyn_smem<n, R>(tpb);
      if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_init_cta<n, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k_init_cta<n, R><<<L.count, tpb, smem, L.stream>>>(L.descs, L.count);
      break;
    }
    case PH_SLR:
      if (qt32) k_slr_cta<n, float, R><<<L.count, tpb, 0, L.stream>>>(L.descs, L.count, arg_i);
      else k_slr_cta<n, double, R><<<L.count, tpb, 0, L.stream>>>(L.descs, L.count, arg_i);
      break;
    case PH_PRIOR: {
      const size_t smem = (size_t)(tpb / 32) * crw::Lay<n>::ws * sizeof(R);
      if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_prior_cta<n, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(k_prior_solve_cta<n, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      k_prior_cta<n, R><<<L.count, tpb, smem, L.stream>>>(L.descs, L.count, arg_i);
      const cudaError_t e0 = cudaGetLastError();
      if (e0 != cudaSuccess) return e0;
      k_prior_solve_cta<n, R><<<L.count, tpb, smem, L.stream>>>(L.descs, L.count);
      break;
    }
    case PH_RELIN: k_relinearised_cta<n, R><<<L.count, tpb, 0, L.stream>>>(L.descs, L.count); break;
    case PH_FINALIZE: k_finalize_cta<n, R><<<L.count, tpb, 0, L.stream>>>(L.descs, L.count); break;
    case PH_WORKING: k_working_cta<n, R><<<L.count, tpb, 0, L.stream>>>(L.descs, L.count); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pgv
