// pgvimp_crw.cuh -- the warp-cooperative cyclic reduction of the block form,
// used for state dimensions n >= 6.
//
// The block form eliminates the states of a plan by block cyclic reduction
// (see pgvimp_cr.cuh for the recurrences).  There, each elimination is one
// thread's n x n block arithmetic on thread-local arrays; for n = 14 those
// arrays (several KB a thread) live in local memory, and from the second level
// on most threads of the block wait at the barrier while a few finish their
// blocks.  Here one WARP performs each elimination: its lanes own the block's
// elements (element e = lane + 32 t), operands are staged in a per-warp slice
// of shared memory, and each block product is n-term dot products, one per
// element.  The arithmetic is the same Thm 1 / natural-gradient trial with the
// same elimination order; differences of rounding order only:
//   * the pivot blocks are inverted by Gauss-Jordan elimination without
//     pivoting (their pivots are the Cholesky pivots of the same SPD block, so
//     positive definiteness and log det are decided from the same Schur
//     complements) and symmetrised from the lower triangle;
//   * double-float block products use a compensated dot product (each product
//     split exactly by the FMA two-product, the leading parts summed by
//     two-sums, every residual collected in FP32, one renormalisation), which
//     is more accurate than a chain of double-float FMAs.
#pragma once
#include "pgvimp_dfx.cuh"
#include "pgvimp_kernels.cuh"

namespace pgv {

// Sum of NV values over the thread block (blockDim.x a multiple of 32); every
// thread receives the same totals (same summation order in every thread).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[w * NV + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int j = 0; j < nw; ++j) s += red[j * NV + k];
    v[k] = s;
  }
}

namespace crw {

// Per-state scratch (R elements, full row-major blocks): working diagonal
// blocks of both systems (their inverses after elimination), couplings, the
// four U blocks, the reduced right-hand side and the mean correction.
// Per-warp shared memory: seven staging blocks, the pivot row and column of
// the inversion, four vectors.
template <int n>
struct Lay {
  static constexpr int nn = n * n;
  static constexpr int oDA = 0, oDM = nn, oCA = 2 * nn, oCM = 3 * nn, oUlA = 4 * nn, oUrA = 5 * nn, oUlM = 6 * nn,
                       oUrM = 7 * nn, oR = 8 * nn, oX = 8 * nn + n;
  static constexpr int stride = 8 * nn + 2 * n;
  static constexpr int nblk = 7;
  static constexpr int oRow = nblk * nn, oCol = oRow + n, oV = oCol + n;
  static constexpr int ws = oV + 4 * n;   // per-warp shared memory, R elements
};

// Dot-product accumulators: an FMA chain in FP64; for double-float the
// compensated sum described at the top of this file.
template <typename R>
struct Acc;
template <>
struct Acc<double> {
  double s;
  PGV_DEV void init(double v) { s = v; }
  PGV_DEV void add(double x, double y) { s = fma(x, y, s); }
  PGV_DEV void merge(const Acc& o) { s += o.s; }
  PGV_DEV double get() const { return s; }
};
template <>
struct Acc<df64> {
  float s, e;
  PGV_DEV void init(df64 v) {
    s = v.hi;
    e = v.lo;
  }
  PGV_DEV void add(df64 x, df64 y) {
    const float p = PGV_FMUL(x.hi, y.hi);
    float q = PGV_FFMA(x.hi, y.hi, -p);
    q = PGV_FFMA(x.hi, y.lo, q);
    q = PGV_FFMA(x.lo, y.hi, q);
    float t, r;
    df_two_sum(s, p, t, r);
    s = t;
    e = PGV_FADD(e, PGV_FADD(r, q));
  }
  PGV_DEV void merge(const Acc& o) {
    float t, r;
    df_two_sum(s, o.s, t, r);
    s = t;
    e = PGV_FADD(e, PGV_FADD(r, o.e));
  }
  PGV_DEV df64 get() const {
    float t, r;
    df_two_sum(s, e, t, r);
    return df_make(t, r);
  }
};

PGV_DEV double neg(double v) { return -v; }
PGV_DEV df64 neg(df64 v) { return df_make(-v.hi, -v.lo); }
// 1/v: IEEE division in FP64, Newton-Raphson steps in double-float (df_rcp).
PGV_DEV double rcp(double v) { return 1.0 / v; }
PGV_DEV df64 rcp(df64 v) { return df_rcp(v); }

// Z = C0 - X' Y' (neg) or C0 + X' Y' over the lane's elements of an n x n
// block, where X' = X or X^T (tx) and Y' = Y or Y^T (ty); C0 null means 0.
// Element e of Z depends on element e of C0 only, so C0 and Z may alias and
// successive calls on the same Z need no synchronisation.  Out of line: one
// copy of the loop serves every product of the sweeps.
template <int n, typename R>
__device__ __noinline__ void mm(int lane, const R* __restrict__ X, const R* __restrict__ Y, const R* C0, R* Z,
                                int tx, int ty, int negate) {
  constexpr int nn = n * n;
  const int sxa = tx ? 1 : n, sxk = tx ? n : 1, syk = ty ? 1 : n, syc = ty ? n : 1;
#pragma unroll 1
  for (int e = lane; e < nn; e += 32) {
    const int a = e / n, c = e - a * n;
    const R* px = X + a * sxa;
    const R* py = Y + c * syc;
    Acc<R> s0, s1;
    R c0 = C0 ? C0[e] : r_fromf<R>(0.0f);
    s0.init(negate ? neg(c0) : c0);
    s1.init(r_fromf<R>(0.0f));
#pragma unroll
    for (int k = 0; k + 1 < n; k += 2) {
      s0.add(px[k * sxk], py[k * syk]);
      s1.add(px[(k + 1) * sxk], py[(k + 1) * syk]);
    }
    if (n & 1) s0.add(px[(n - 1) * sxk], py[(n - 1) * syk]);
    s0.merge(s1);
    const R z = s0.get();
    Z[e] = negate ? neg(z) : z;
  }
}

// y = y0 - M' v (neg) or y0 + M' v for the n entries (lanes 0..n-1), M' = M
// or M^T; y0 null means 0; y may alias y0.
template <int n, typename R>
PGV_DEV void mv(int lane, const R* M, bool tm, const R* v, const R* y0, R* y, bool negate) {
  if (lane < n) {
    Acc<R> s;
    R c0 = y0 ? y0[lane] : r_fromf<R>(0.0f);
    s.init(negate ? neg(c0) : c0);
#pragma unroll
    for (int k = 0; k < n; ++k) s.add(tm ? M[k * n + lane] : M[lane * n + k], v[k]);
    const R z = s.get();
    y[lane] = negate ? neg(z) : z;
  }
}

template <int n, typename R>
PGV_DEV void wcopy(int lane, R* dst, const R* src) {
#pragma unroll 1
  for (int e = lane; e < n * n; e += 32) dst[e] = src[e];
}

// In-place inverse of the symmetric positive definite block S (shared
// memory) by Gauss-Jordan elimination; pivot k is the leading entry of the
// k-th Schur complement.  `ok` is cleared unless every pivot is > 0 (a
// non-positive pivot is replaced by 1 so that the sweep stays finite; the
// trial is then rejected); the pivots feed `ld`.  The result is symmetrised
// from its lower triangle.
template <int n, typename R>
PGV_DEV void winv(int lane, R* S, R* row, R* col, LogDetAcc<R>& ld, bool& ok) {
  constexpr int nn = n * n, EPL = (nn + 31) / 32;
  const R one = r_fromf<R>(1.0f);
  __syncwarp();
#pragma unroll 1
  for (int k = 0; k < n; ++k) {
    if (lane < n) {
      row[lane] = S[k * n + lane];
      col[lane] = S[lane * n + k];
    }
    __syncwarp();
    R p = row[k];
    ok = ok && r_pos(p);
    p = r_pos(p) ? p : one;
    ld.mul(p);
    const R ip = rcp(p);
    R nv[EPL];
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
      const int e = lane + 32 * t;
      if (e < nn) {
        const int a = e / n, c = e - a * n;
        const R rk = row[c], ck = col[a];
        const R tk = rk * ip;
        nv[t] = (a == k) ? ((c == k) ? ip : tk) : ((c == k) ? neg(ck * ip) : r_fma(neg(ck), tk, S[e]));
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < EPL; ++t) {
      const int e = lane + 32 * t;
      if (e < nn) S[e] = nv[t];
    }
    __syncwarp();
  }
  R nv[EPL];
#pragma unroll
  for (int t = 0; t < EPL; ++t) {
    const int e = lane + 32 * t;
    if (e < nn) {
      const int a = e / n, c = e - a * n;
      nv[t] = S[a >= c ? e : c * n + a];
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < EPL; ++t) {
    const int e = lane + 32 * t;
    if (e < nn) S[e] = nv[t];
  }
  __syncwarp();
}

// Store of a block (shared memory) to memory symmetrised from its lower
// triangle; dst and src do not alias.
template <int n, typename R>
PGV_DEV void wst_sym(int lane, R* dst, const R* src) {
#pragma unroll 1
  for (int e = lane; e < n * n; e += 32) {
    const int a = e / n, c = e - a * n;
    dst[e] = src[a >= c ? e : c * n + a];
  }
}

// Thm 1 (or the natural-gradient step) at step beta by cyclic reduction with
// one warp per elimination; the same scaled system, outputs and TrialOut as
// cr_trial.  `wsm` is this block's dynamic shared memory (Lay::ws elements a
// warp).
template <int n, typename R>
PGV_BIG TrialOut trial(const PlanDesc& P, double beta_d, int cur, int out, double logdet_k, bool marg_only,
                       double* red, R* wsm) {
  using Ly = Lay<n>;
  constexpr int nn = n * n, SS = Ly::stride;
  const int N = P.N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  R* ws = wsm + (size_t)warp * Ly::ws;
  R* S0 = ws;
  R* S1 = ws + nn;
  R* S2 = ws + 2 * nn;
  R* S3 = ws + 3 * nn;
  R* S4 = ws + 4 * nn;
  R* S5 = ws + 5 * nn;
  R* S6 = ws + 6 * nn;
  R* row = ws + Ly::oRow;
  R* col = ws + Ly::oCol;
  R* V0 = ws + Ly::oV;
  R* V1 = V0 + n;
  R* V2 = V1 + n;
  R* V3 = V2 + n;
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
  const bool ngd = wm && (P.update == PGVIMP_UPDATE_NGD);
  const R cL = ngd ? r_from<R>(1.0 - beta_d) : r_fromf<R>(1.0f);
  TrialOut res;
  res.kl = INFINITY;
  res.pd = false;
  res.logdet = 0.0;
  res.prior_cost = 0.0;
  res.delta = 0.0;
  res.trace = 0.0;

  // ---- level-0 system: warps over states, lanes over block elements
  for (int i = warp; i <= N; i += NW) {
    R* sp = scr + (size_t)i * SS;
    const size_t oi = (size_t)i * nn;
#pragma unroll 1
    for (int e = lane; e < nn; e += 32) {
      R L = Ld[oi + e];
      if (ngd) L = cL * L;
      R DA = L;
      if (wm) {
        const R K = Kd[oi + e], G = GG[oi + e];
        const R kb = beta * K;
        R DM = L + kb;
        if (ngd) DM = r_fma(beta2, G, DM);
        DA = r_fma(beta2, G, L + kb);
        sp[Ly::oDM + e] = DM;
      }
      sp[Ly::oDA + e] = DA;
      if (i < N) {
        R E = Lo[oi + e];
        if (ngd) E = cL * E;
        if (wm) {
          E = r_fma(beta, Ko[oi + e], E);   // beta K^-1_{i+1,i} + c Lambda_{i+1,i}
          sp[Ly::oCM + e] = E;
        }
        sp[Ly::oCA + e] = E;
      }
    }
    if (wm && lane < n) {
      // rhs_i = beta (b_i - g_i - (K^-1 mu)_i)
      const int a = lane;
      Acc<R> s;
      s.init(zero);
      for (int c = 0; c < n; ++c) s.add(Kd[oi + a * n + c], mu[(size_t)i * n + c]);
      if (i > 0)
        for (int c = 0; c < n; ++c) s.add(Ko[oi - nn + a * n + c], mu[(size_t)(i - 1) * n + c]);
      if (i < N)
        for (int c = 0; c < n; ++c) s.add(Ko[oi + c * n + a], mu[(size_t)(i + 1) * n + c]);
      sp[Ly::oR + a] = beta * ((bb[(size_t)i * n + a] - gg[(size_t)i * n + a]) - s.get());
    }
  }
  __syncthreads();

  // ---- forward: eliminate the odd multiples of h, one warp per state
  LogDetAcc<R> ldA, ldM;
  ldA.init();
  ldM.init();
  bool okA = true, okM = true;
  int h = 1;
  for (; h <= N; h <<= 1) {
    for (int i = h + 2 * h * warp; i <= N; i += 2 * h * NW) {
      R* sp = scr + (size_t)i * SS;
      const R* spl = scr + (size_t)(i - h) * SS;
      const bool hasr = (i + h <= N);
      wcopy<n, R>(lane, S0, sp + Ly::oDA);
      wcopy<n, R>(lane, S1, spl + Ly::oCA);                 // A_{i,l}
      if (hasr) wcopy<n, R>(lane, S2, sp + Ly::oCA);        // A_{r,i}; A_{i,r} is its transpose
      if (wm) {
        wcopy<n, R>(lane, S3, sp + Ly::oDM);
        wcopy<n, R>(lane, S4, spl + Ly::oCM);
        if (hasr) wcopy<n, R>(lane, S5, sp + Ly::oCM);
        if (lane < n) V0[lane] = sp[Ly::oR + lane];
      }
      winv<n, R>(lane, S0, row, col, ldA, okA);             // D_i^-1 (ends with __syncwarp)
      wcopy<n, R>(lane, sp + Ly::oDA, S0);
      mm<n, R>(lane, S0, S1, nullptr, sp + Ly::oUlA, 0, 0, 0);              // U_l = D^-1 A_{i,l}
      if (hasr) mm<n, R>(lane, S0, S2, nullptr, sp + Ly::oUrA, 0, 1, 0);    // U_r = D^-1 A_{r,i}^T
      if (wm) {
        winv<n, R>(lane, S3, row, col, ldM, okM);
        wcopy<n, R>(lane, sp + Ly::oDM, S3);
        mm<n, R>(lane, S3, S4, nullptr, sp + Ly::oUlM, 0, 0, 0);
        if (hasr) mm<n, R>(lane, S3, S5, nullptr, sp + Ly::oUrM, 0, 1, 0);
        mv<n, R>(lane, S3, false, V0, nullptr, sp + Ly::oR, false);        // y_i = D^-1 rhs_i
      }
      __syncwarp();
    }
    __syncthreads();
    // survivors j (multiples of 2h): Schur updates from j - h and j + h
    for (int j = 2 * h * warp; j <= N; j += 2 * h * NW) {
      R* sp = scr + (size_t)j * SS;
      const bool hasl = (j >= h), hasr = (j + h <= N), has2 = (j + 2 * h <= N);
      const R* spl = scr + (size_t)(hasl ? j - h : j) * SS;
      const R* spr = scr + (size_t)(hasr ? j + h : j) * SS;
#pragma unroll 1
      for (int sys = 0; sys < (wm ? 2 : 1); ++sys) {
        const int oD = sys ? Ly::oDM : Ly::oDA, oC = sys ? Ly::oCM : Ly::oCA;
        const int oUl = sys ? Ly::oUlM : Ly::oUlA, oUr = sys ? Ly::oUrM : Ly::oUrA;
        if (hasl) {
          wcopy<n, R>(lane, S0, spl + oC);                  // A_{j,i}, i = j - h
          wcopy<n, R>(lane, S1, spl + oUr);
        }
        if (hasr) {
          wcopy<n, R>(lane, S2, sp + oC);                   // A_{i,j}, i = j + h
          wcopy<n, R>(lane, S3, spr + oUl);
          if (has2) wcopy<n, R>(lane, S4, spr + oC);        // A_{j+2h,i}
        }
        if (sys && lane < n) {
          V0[lane] = sp[Ly::oR + lane];
          if (hasl) V1[lane] = spl[Ly::oR + lane];
          if (hasr) V2[lane] = spr[Ly::oR + lane];
        }
        __syncwarp();
        if (hasl) mm<n, R>(lane, S0, S1, sp + oD, sp + oD, 0, 0, 1);          // D_j -= A_{j,i} U_r(i)
        if (hasr) {
          mm<n, R>(lane, S2, S3, sp + oD, sp + oD, 1, 0, 1);                  // D_j -= A_{i,j}^T U_l(i)
          if (has2) mm<n, R>(lane, S4, S3, nullptr, sp + oC, 0, 0, 1);        // A_{j+2h,j} = -A_{j+2h,i} U_l(i)
        }
        if (sys) {
          if (hasl) mv<n, R>(lane, S0, false, V1, V0, V0, true);              // r_j -= A_{j,i} y_i
          if (hasr) mv<n, R>(lane, S2, true, V2, V0, V0, true);               // r_j -= A_{i,j}^T y_i
          if (lane < n) sp[Ly::oR + lane] = V0[lane];
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  // ---- root (state 0)
  if (warp == 0) {
    wcopy<n, R>(lane, S0, scr + Ly::oDA);
    if (wm) {
      wcopy<n, R>(lane, S3, scr + Ly::oDM);
      if (lane < n) V0[lane] = scr[Ly::oR + lane];
    }
    winv<n, R>(lane, S0, row, col, ldA, okA);
    wcopy<n, R>(lane, Sd_out, S0);
    if (wm) {
      winv<n, R>(lane, S3, row, col, ldM, okM);
      mv<n, R>(lane, S3, false, V0, nullptr, scr + Ly::oX, false);
    }
  }
  const bool pd = __syncthreads_and(okA && okM);
  double lsum[1] = {lane == 0 ? ldA.log_value() : 0.0};   // the accumulator is uniform over the warp
  block_sum<1>(lsum, red);
  if (!pd) return res;

  // ---- backward: selected inverse and back substitution, top level first
  for (h >>= 1; h >= 1; h >>= 1) {
    for (int i = h + 2 * h * warp; i <= N; i += 2 * h * NW) {
      const int l = i - h, r = i + h;
      const bool hasr = (r <= N);
      const R* sp = scr + (size_t)i * SS;
      wcopy<n, R>(lane, S0, Sd_out + (size_t)l * nn);       // Sigma_ll
      wcopy<n, R>(lane, S1, sp + Ly::oUlA);                 // U_l
      if (hasr) {
        wcopy<n, R>(lane, S2, So_out + (size_t)l * nn);     // Sigma_{r,l}
        wcopy<n, R>(lane, S3, Sd_out + (size_t)r * nn);     // Sigma_rr
        wcopy<n, R>(lane, S4, sp + Ly::oUrA);               // U_r
      }
      if (wm && lane < n) {
        V0[lane] = sp[Ly::oR + lane];
        V1[lane] = scr[(size_t)l * SS + Ly::oX + lane];
        if (hasr) V2[lane] = scr[(size_t)r * SS + Ly::oX + lane];
      }
      __syncwarp();
      mm<n, R>(lane, S1, S0, nullptr, S5, 0, 0, 1);                           // Sigma_il = -U_l Sigma_ll
      if (hasr) {
        mm<n, R>(lane, S4, S2, S5, S5, 0, 0, 1);                              //            - U_r Sigma_rl
        mm<n, R>(lane, S4, S3, nullptr, S6, 0, 0, 1);                         // Sigma_ir = -U_r Sigma_rr
        mm<n, R>(lane, S1, S2, S6, S6, 0, 1, 1);                              //            - U_l Sigma_lr
      }
      __syncwarp();
      mm<n, R>(lane, S5, S1, sp + Ly::oDA, S0, 0, 1, 1);                      // Sigma_ii = D^-1 - Sigma_il U_l^T
      if (hasr) mm<n, R>(lane, S6, S4, S0, S0, 0, 1, 1);                      //            - Sigma_ir U_r^T
      __syncwarp();
      wst_sym<n, R>(lane, Sd_out + (size_t)i * nn, S0);
      wcopy<n, R>(lane, So_out + (size_t)l * nn, S5);       // Sigma_{i,l} = Sigma_{l+h,l}
      if (hasr) {
#pragma unroll 1
        for (int e = lane; e < nn; e += 32) {
          const int a = e / n, c = e - a * n;
          So_out[(size_t)i * nn + e] = S6[c * n + a];       // Sigma_{r,i} = Sigma_ir^T
        }
      }
      if (wm) {
        // x_i = y_i - U_l^M x_l - U_r^M x_r
        wcopy<n, R>(lane, S1, sp + Ly::oUlM);
        if (hasr) wcopy<n, R>(lane, S4, sp + Ly::oUrM);
        __syncwarp();
        mv<n, R>(lane, S1, false, V1, V0, V0, true);
        if (hasr) mv<n, R>(lane, S4, false, V2, V0, V0, true);
        if (lane < n) scr[(size_t)i * SS + Ly::oX + lane] = V0[lane];
      }
      __syncwarp();
    }
    __syncthreads();
  }

  // ---- KL pieces, prior cost, outputs scaled by s (beta + 1, or 1 for the natural-gradient step)
  const double bp1d = ngd ? 1.0 : beta_d + 1.0;
  const R bp1 = r_from<R>(bp1d);
  R trc = zero, dl = zero, ktr = zero, kq = zero;
  for (int i = warp; i <= N; i += NW) {
    const size_t oi = (size_t)i * nn;
    if (lane < n) {
      const int a = lane;
      const R xi = wm ? scr[(size_t)i * SS + Ly::oX + a] : zero;
      const R mo = mu[(size_t)i * n + a] + xi;
      V0[a] = xi;
      V1[a] = mo - mubar[(size_t)i * n + a];
      if (wm) mo_out[(size_t)i * n + a] = mo;
      if (i < N) {
        const R xn = wm ? scr[(size_t)(i + 1) * SS + Ly::oX + a] : zero;
        V2[a] = xn;
        V3[a] = (mu[(size_t)(i + 1) * n + a] + xn) - mubar[(size_t)(i + 1) * n + a];
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int e = lane; e < nn; e += 32) {
      const int a = e / n, c = e - a * n;
      const R Si = Sd_out[oi + e];
      if (wm) {
        const R B = Ld[oi + e], G = GG[oi + e];
        trc = r_fma(B, Si, trc);
        dl = r_fma(V0[a] * B, V0[c], dl);
        trc = r_fma(neg(G + G), Si, trc);
      }
      const R K = Kd[oi + e];
      trc = r_fma(neg(K), Si, trc);
      ktr = r_fma(K, Si, ktr);
      kq = r_fma(V1[a] * K, V1[c], kq);
      if (i < N) {
        const R So = So_out[oi + e];   // Sigma~_{i+1,i}
        if (wm) {
          const R B = Lo[oi + e];
          trc = r_fma(B + B, So, trc);
          dl = r_fma((V2[a] + V2[a]) * B, V0[c], dl);
        }
        const R Kb = Ko[oi + e];
        trc = r_fma(neg(Kb + Kb), So, trc);
        ktr = r_fma(Kb + Kb, So, ktr);
        kq = r_fma((V3[a] + V3[a]) * Kb, V1[c], kq);
        if (wm) So_out[oi + e] = bp1 * So;
      }
      if (wm) Sd_out[oi + e] = bp1 * Si;
    }
    __syncwarp();
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

// x = M^-1 r for the symmetric positive definite block tridiagonal M with
// diagonal blocks Md and sub-diagonal blocks Mo (block (i+1, i) at Mo + i n^2),
// by the same warp-cooperative cyclic reduction (the mean system of `trial`
// alone).  Uses the plan's scratch.  Every thread returns whether every pivot
// was positive (x is written only then).
template <int n, typename R>
PGV_BIG bool solve(const PlanDesc& P, const R* Md, const R* Mo, const R* r, R* x, R* wsm) {
  using Ly = Lay<n>;
  constexpr int nn = n * n, SS = Ly::stride;
  const int N = P.N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
  R* ws = wsm + (size_t)warp * Ly::ws;
  R* S0 = ws;
  R* S1 = ws + nn;
  R* S2 = ws + 2 * nn;
  R* S3 = ws + 3 * nn;
  R* S4 = ws + 4 * nn;
  R* row = ws + Ly::oRow;
  R* col = ws + Ly::oCol;
  R* V0 = ws + Ly::oV;
  R* V1 = V0 + n;
  R* V2 = V1 + n;
  R* scr = rp<R>(P.scr);
  for (int i = warp; i <= N; i += NW) {
    R* sp = scr + (size_t)i * SS;
#pragma unroll 1
    for (int e = lane; e < nn; e += 32) {
      sp[Ly::oDM + e] = Md[(size_t)i * nn + e];
      if (i < N) sp[Ly::oCM + e] = Mo[(size_t)i * nn + e];
    }
    if (lane < n) sp[Ly::oR + lane] = r[(size_t)i * n + lane];
  }
  __syncthreads();
  LogDetAcc<R> ld;
  ld.init();
  bool ok = true;
  int h = 1;
  for (; h <= N; h <<= 1) {
    for (int i = h + 2 * h * warp; i <= N; i += 2 * h * NW) {
      R* sp = scr + (size_t)i * SS;
      const R* spl = scr + (size_t)(i - h) * SS;
      const bool hasr = (i + h <= N);
      wcopy<n, R>(lane, S0, sp + Ly::oDM);
      wcopy<n, R>(lane, S1, spl + Ly::oCM);
      if (hasr) wcopy<n, R>(lane, S2, sp + Ly::oCM);
      if (lane < n) V0[lane] = sp[Ly::oR + lane];
      winv<n, R>(lane, S0, row, col, ld, ok);
      mm<n, R>(lane, S0, S1, nullptr, sp + Ly::oUlM, 0, 0, 0);
      if (hasr) mm<n, R>(lane, S0, S2, nullptr, sp + Ly::oUrM, 0, 1, 0);
      mv<n, R>(lane, S0, false, V0, nullptr, sp + Ly::oR, false);
      __syncwarp();
    }
    __syncthreads();
    for (int j = 2 * h * warp; j <= N; j += 2 * h * NW) {
      R* sp = scr + (size_t)j * SS;
      const bool hasl = (j >= h), hasr = (j + h <= N), has2 = (j + 2 * h <= N);
      const R* spl = scr + (size_t)(hasl ? j - h : j) * SS;
      const R* spr = scr + (size_t)(hasr ? j + h : j) * SS;
      if (hasl) {
        wcopy<n, R>(lane, S0, spl + Ly::oCM);
        wcopy<n, R>(lane, S1, spl + Ly::oUrM);
      }
      if (hasr) {
        wcopy<n, R>(lane, S2, sp + Ly::oCM);
        wcopy<n, R>(lane, S3, spr + Ly::oUlM);
        if (has2) wcopy<n, R>(lane, S4, spr + Ly::oCM);
      }
      if (lane < n) {
        V0[lane] = sp[Ly::oR + lane];
        if (hasl) V1[lane] = spl[Ly::oR + lane];
        if (hasr) V2[lane] = spr[Ly::oR + lane];
      }
      __syncwarp();
      if (hasl) mm<n, R>(lane, S0, S1, sp + Ly::oDM, sp + Ly::oDM, 0, 0, 1);
      if (hasr) {
        mm<n, R>(lane, S2, S3, sp + Ly::oDM, sp + Ly::oDM, 1, 0, 1);
        if (has2) mm<n, R>(lane, S4, S3, nullptr, sp + Ly::oCM, 0, 0, 1);
      }
      if (hasl) mv<n, R>(lane, S0, false, V1, V0, V0, true);
      if (hasr) mv<n, R>(lane, S2, true, V2, V0, V0, true);
      if (lane < n) sp[Ly::oR + lane] = V0[lane];
      __syncwarp();
    }
    __syncthreads();
  }
  if (warp == 0) {
    wcopy<n, R>(lane, S0, scr + Ly::oDM);
    if (lane < n) V0[lane] = scr[Ly::oR + lane];
    winv<n, R>(lane, S0, row, col, ld, ok);
    mv<n, R>(lane, S0, false, V0, nullptr, scr + Ly::oX, false);
  }
  if (!__syncthreads_and(ok)) return false;
  for (h >>= 1; h >= 1; h >>= 1) {
    for (int i = h + 2 * h * warp; i <= N; i += 2 * h * NW) {
      const int l = i - h, rr = i + h;
      const bool hasr = (rr <= N);
      const R* sp = scr + (size_t)i * SS;
      wcopy<n, R>(lane, S1, sp + Ly::oUlM);
      if (hasr) wcopy<n, R>(lane, S4, sp + Ly::oUrM);
      if (lane < n) {
        V0[lane] = sp[Ly::oR + lane];
        V1[lane] = scr[(size_t)l * SS + Ly::oX + lane];
        if (hasr) V2[lane] = scr[(size_t)rr * SS + Ly::oX + lane];
      }
      __syncwarp();
      mv<n, R>(lane, S1, false, V1, V0, V0, true);
      if (hasr) mv<n, R>(lane, S4, false, V2, V0, V0, true);
      if (lane < n) scr[(size_t)i * SS + Ly::oX + lane] = V0[lane];
      __syncwarp();
    }
    __syncthreads();
  }
  for (int i = warp; i <= N; i += NW)
    if (lane < n) x[(size_t)i * n + lane] = scr[(size_t)i * SS + Ly::oX + lane];
  __syncthreads();
  return true;
}

// Lambda_{k+1} = A~(beta) / s over (Ld, Lo), element-parallel over the block.
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
  const size_t nd = (size_t)(N + 1) * nn, no = (size_t)N * nn;
  for (size_t e = threadIdx.x; e < nd; e += blockDim.x) Ld[e] = r_fma(beta, r_fma(two, GG[e], Kd[e]), cL * Ld[e]) * inv;
  for (size_t e = threadIdx.x; e < no; e += blockDim.x) Lo[e] = r_fma(beta, Ko[e], cL * Lo[e]) * inv;
}

}  // namespace crw
}  // namespace pgv
