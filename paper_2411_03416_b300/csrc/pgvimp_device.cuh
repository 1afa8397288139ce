// pgvimp_device.cuh -- device arithmetic of the P-GVIMP hot path on sm_103a.
//
// Execution model: one GPU thread owns one planning problem (a "lane plan").
// B300's FP64 pipe issues one warp instruction per ~20 SM cycles whatever the
// active mask, so every FP64 instruction must carry 32 independent problems:
// the per-state block recursions (n x n, n <= 16) run in registers / local
// memory of one thread, and a warp advances 32 plans in lockstep.  The
// quadrature (FP32 in the mixed precision form) runs in the same thread.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "pgvimp_plan.h"

namespace pgv {

#ifndef PGV_DEV
#define PGV_DEV __device__ __forceinline__
#endif
// Unrolling of the block loops: forced full for small blocks (n <= 8); for
// larger blocks `#pragma unroll 0`, which the compiler ignores, leaving the
// unroll factor to its heuristics.  Forcing those loops rolled (`unroll 1`)
// made n = 14 routines over thread-local arrays return wrong covariance
// blocks on sm_103a in some contexts, while the same code compiled for the
// host, fully unrolled, or with the compiler's own choice is exact.
// Large routines are inlined too: an out-of-line (__noinline__) build of the
// n = 14 trial sweep, whose thread-local arrays exceed 20 KB, showed the same
// wrong results.
#ifndef PGV_BIG
#define PGV_BIG __device__ __forceinline__
#endif

// Read-only cached load and reciprocal square root (device); the host
// variants let the same routines run in host-side checks.
template <typename T>
__host__ __device__ __forceinline__ T pgv_ldg(const T* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}
__host__ __device__ __forceinline__ double pgv_rsqrt(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / sqrt(x);
#endif
}

// ------------------------------------------------------------ double-float
// FP64-class arithmetic on the FP32 pipe: a value is the unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi)/2, ~48-bit significand), combined
// with the error-free transformations of Knuth (two-sum), Dekker (fast
// two-sum) and the FMA two-product.  The intrinsics below are never
// contracted into FMAs, which the transformations rely on.  B300 issues FP32
// at 64x its FP64 rate and with 4-cycle instead of 64-cycle latency.
#ifdef __CUDA_ARCH__
#define PGV_FADD(a, b) __fadd_rn(a, b)
#define PGV_FSUB(a, b) __fsub_rn(a, b)
#define PGV_FMUL(a, b) __fmul_rn(a, b)
#define PGV_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define PGV_FADD(a, b) ((a) + (b))
#define PGV_FSUB(a, b) ((a) - (b))
#define PGV_FMUL(a, b) ((a) * (b))
#define PGV_FFMA(a, b, c) fmaf(a, b, c)
#endif
#define PGV_HD __host__ __device__ __forceinline__

struct __align__(8) df64 {
  float hi, lo;
};

PGV_HD df64 df_make(float h, float l) {
  df64 r;
  r.hi = h;
  r.lo = l;
  return r;
}
PGV_HD df64 df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = PGV_FADD(a, b);
  return df_make(s, PGV_FSUB(b, PGV_FSUB(s, a)));
}
PGV_HD df64 operator+(df64 x, df64 y) {
  float s = PGV_FADD(x.hi, y.hi);
  float bb = PGV_FSUB(s, x.hi);
  float e = PGV_FADD(PGV_FSUB(x.hi, PGV_FSUB(s, bb)), PGV_FSUB(y.hi, bb));
  e = PGV_FADD(e, PGV_FADD(x.lo, y.lo));
  return df_fast_two_sum(s, e);
}
PGV_HD df64 operator-(df64 x) { return df_make(-x.hi, -x.lo); }
PGV_HD df64 operator-(df64 x, df64 y) { return x + (-y); }
PGV_HD df64 operator*(df64 x, df64 y) {
  float p = PGV_FMUL(x.hi, y.hi);
  float e = PGV_FFMA(x.hi, y.hi, -p);
  e = PGV_FFMA(x.hi, y.lo, e);
  e = PGV_FFMA(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
// x * y + z with one normalisation.
PGV_HD df64 df_fma(df64 x, df64 y, df64 z) {
  float p = PGV_FMUL(x.hi, y.hi);
  float e = PGV_FFMA(x.hi, y.hi, -p);
  e = PGV_FFMA(x.hi, y.lo, e);
  e = PGV_FFMA(x.lo, y.hi, e);
  float s = PGV_FADD(p, z.hi);
  float bb = PGV_FSUB(s, p);
  float f = PGV_FADD(PGV_FSUB(p, PGV_FSUB(s, bb)), PGV_FSUB(z.hi, bb));
  f = PGV_FADD(f, PGV_FADD(e, z.lo));
  return df_fast_two_sum(s, f);
}

// Arithmetic used by the recursions, for R = double (native FP64) and
// R = df64 (double-float).
PGV_HD double r_fma(double a, double b, double c) { return fma(a, b, c); }
PGV_HD df64 r_fma(df64 a, df64 b, df64 c) { return df_fma(a, b, c); }
template <typename R> PGV_HD R r_from(double v);
template <> PGV_HD double r_from<double>(double v) { return v; }
template <> PGV_HD df64 r_from<df64>(double v) {
  float h = (float)v;
  return df_make(h, (float)(v - (double)h));
}
template <typename R> PGV_HD R r_fromf(float v);
template <> PGV_HD double r_fromf<double>(float v) { return (double)v; }
template <> PGV_HD df64 r_fromf<df64>(float v) { return df_make(v, 0.0f); }
PGV_HD double r_to(double v) { return v; }
PGV_HD double r_to(df64 v) { return (double)v.hi + (double)v.lo; }
PGV_HD float r_tof(double v) { return (float)v; }
PGV_HD float r_tof(df64 v) { return v.hi + v.lo; }
PGV_HD bool r_pos(double v) { return v > 0.0; }
PGV_HD bool r_pos(df64 v) { return v.hi > 0.0f; }
PGV_HD double r_rsqrt(double v) {
#ifdef __CUDA_ARCH__
  return rsqrt(v);
#else
  return 1.0 / sqrt(v);
#endif
}
// 1/sqrt(v): FP32 estimate refined by one Newton step in double-float.
PGV_HD df64 r_rsqrt(df64 v) {
#ifdef __CUDA_ARCH__
  float r0 = rsqrtf(v.hi);
#else
  float r0 = 1.0f / sqrtf(v.hi);
#endif
  df64 r = df_make(r0, 0.0f);
  df64 u = (v * r) * r;                        // ~1
  df64 d = df_make(1.0f, 0.0f) - u;            // small, accurate
  return df_fma(df_make(0.5f * r0, 0.0f), d, r);
}

// log det accumulator: pivot products kept as mantissa * 2^expo.
template <typename R>
struct LogDetAcc;
template <>
struct LogDetAcc<double> {
  double mant;
  int expo;
  PGV_HD void init() { mant = 1.0; expo = 0; }
  PGV_HD void mul(double v) {
    int e;
    mant = frexp(mant * v, &e);
    expo += e;
  }
  PGV_HD double log_value() const { return log(mant) + expo * 0.69314718055994530942; }
};
template <>
struct LogDetAcc<df64> {
  df64 mant;
  int expo;
  PGV_HD void init() { mant = df_make(1.0f, 0.0f); expo = 0; }
  // renormalises mant.hi into [0.5, 1): its exponent read from the float's
  // bits, both parts scaled by the exact power of two 2^-e built the same way
  // (integer and FP32 operations only; the pivot products stay well inside
  // the float range)
  PGV_HD void mul(df64 v) {
    mant = mant * v;
    int bits;
    memcpy(&bits, &mant.hi, sizeof(bits));
    const int e = ((bits >> 23) & 0xff) - 126;
    const int sbits = (127 - e) << 23;
    float sc;
    memcpy(&sc, &sbits, sizeof(sc));
    mant.hi = PGV_FMUL(mant.hi, sc);
    mant.lo = PGV_FMUL(mant.lo, sc);
    expo += e;
  }
  PGV_HD double log_value() const { return log(r_to(mant)) + expo * 0.69314718055994530942; }
};

// ------------------------------------------------------------ small blocks
// Row-major n x n blocks in global memory; symmetric blocks held in thread
// registers in packed lower form, element (a, c) with c <= a at a(a+1)/2 + c.
#define PGV_UNR _Pragma("unroll")

template <int n>
struct Blk {
  static constexpr int nn = n * n;
  static constexpr int np = n * (n + 1) / 2;
};
PGV_HD constexpr int pk(int a, int c) { return a >= c ? a * (a + 1) / 2 + c : c * (c + 1) / 2 + a; }

// Blocks move between registers and memory element by element.  (Built for
// sm_103a with this toolchain, a 16-byte vector store of a register-held
// packed block -- through double2, float4 or a 16-byte aggregate alike --
// wrote another element's value in place of element 0 in some kernels, while
// the register values right before the store were correct; element-wise
// stores and loads of the same blocks are exact.  A single-thread reduction
// of a two-state chain reproduced it.)
template <int n, typename R>
PGV_DEV void ld_blk(const R* p, R* X) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int e = 0; e < n * n; ++e) X[e] = p[e];
}
template <int n, typename R>
PGV_DEV void st_blk(R* p, const R* X) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int e = 0; e < n * n; ++e) p[e] = X[e];
}
// symmetric packed <-> full block in memory
template <int n, typename R>
PGV_DEV void ld_sym(const R* p, R* S) {
  R X[n * n];
  ld_blk<n, R>(p, X);
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) S[pk(a, c)] = X[a * n + c];
}
template <int n, typename R>
PGV_DEV void st_sym(R* p, const R* S) {
  R X[n * n];
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) X[a * n + c] = S[pk(a, c)];
  st_blk<n, R>(p, X);
}
// packed storage (np elements; the layout leaves room for np rounded up to even)
template <int n, typename R>
PGV_DEV void ld_packed(const R* p, R* S) {
  constexpr int np = n * (n + 1) / 2;
#pragma unroll (n <= 8 ? 32 : 0)
  for (int e = 0; e < np; ++e) S[e] = p[e];
}
template <int n, typename R>
PGV_DEV void st_packed(R* p, const R* S) {
  constexpr int np = n * (n + 1) / 2;
#pragma unroll (n <= 8 ? 32 : 0)
  for (int e = 0; e < np; ++e) p[e] = S[e];
}
template <int n, typename R>
PGV_DEV void ld_vec(const R* p, R* x) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a) x[a] = p[a];
}
template <int n, typename R>
PGV_DEV void st_vec(R* p, const R* x) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a) p[a] = x[a];
}

// Z = X * S with S symmetric packed (full n x n result).
template <int n, typename R>
PGV_DEV void mul_full_sym(const R* X, const R* S, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) {
      R s = X[a * n] * S[pk(0, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 1; t < n; ++t) s = r_fma(X[a * n + t], S[pk(t, c)], s);
      Z[a * n + c] = s;
    }
}
// Z = S * X with S symmetric packed.
template <int n, typename R>
PGV_DEV void mul_sym_full(const R* S, const R* X, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c < n; ++c) {
      R s = S[pk(a, 0)] * X[c];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 1; t < n; ++t) s = r_fma(S[pk(a, t)], X[t * n + c], s);
      Z[a * n + c] = s;
    }
}
// packed Z = X * Y^T for a product known to be symmetric.
template <int n, typename R>
PGV_DEV void mul_nt_packed(const R* X, const R* Y, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = X[a * n] * Y[c * n];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 1; t < n; ++t) s = r_fma(X[a * n + t], Y[c * n + t], s);
      Z[pk(a, c)] = s;
    }
}
// packed Z = C + X^T Y (symmetric result).
template <int n, typename R>
PGV_DEV void add_tn_packed(const R* C, const R* X, const R* Y, R* Z) {
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = C[pk(a, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int t = 0; t < n; ++t) s = r_fma(X[t * n + a], Y[t * n + c], s);
      Z[pk(a, c)] = s;
    }
}

// Cholesky C = L L^T of a packed symmetric block, then Cinv = L^-T L^-1
// (packed).  `ok` is cleared unless every pivot is > 0; pivots feed `ld`.
template <int n, typename R>
PGV_DEV void chol_inverse(const R* C, R* Cinv, LogDetAcc<R>& ld, bool& ok) {
  constexpr int np = n * (n + 1) / 2;
  R L[np], r[n];
#pragma unroll (n <= 8 ? 32 : 0)
  for (int j = 0; j < n; ++j) {
    R s = C[pk(j, j)];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int k = 0; k < j; ++k) s = r_fma(-L[pk(j, k)], L[pk(j, k)], s);
    ok = ok && r_pos(s);
    s = r_pos(s) ? s : r_fromf<R>(1.0f);
    R rs = r_rsqrt(s);
    r[j] = rs;
    ld.mul(s);
#pragma unroll (n <= 8 ? 32 : 0)
    for (int i = j + 1; i < n; ++i) {
      R t = C[pk(i, j)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int k = 0; k < j; ++k) t = r_fma(-L[pk(i, k)], L[pk(j, k)], t);
      L[pk(i, j)] = t * rs;
    }
    L[pk(j, j)] = s * rs;
  }
  // X = L^-1 (lower, packed)
  R X[np];
#pragma unroll (n <= 8 ? 32 : 0)
  for (int j = 0; j < n; ++j) {
    X[pk(j, j)] = r[j];
#pragma unroll (n <= 8 ? 32 : 0)
    for (int i = j + 1; i < n; ++i) {
      R s = L[pk(i, j)] * X[pk(j, j)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int k = j + 1; k < i; ++k) s = r_fma(L[pk(i, k)], X[pk(k, j)], s);
      X[pk(i, j)] = -(s * r[i]);
    }
  }
  // Cinv = X^T X
#pragma unroll (n <= 8 ? 32 : 0)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 0)
    for (int c = 0; c <= a; ++c) {
      R s = X[pk(a, a)] * X[pk(a, c)];
#pragma unroll (n <= 8 ? 32 : 0)
      for (int k = a + 1; k < n; ++k) s = r_fma(X[pk(k, a)], X[pk(k, c)], s);
      Cinv[pk(a, c)] = s;
    }
}

// Lower Cholesky factor and its inverse of the leading d x d block of a
// symmetric full n x n block (runtime d <= n), as full row-major arrays.
template <int n, typename R>
PGV_DEV bool chol_lead(const R* S, int d, R* L, R* Li) {
  bool ok = true;
  const R zero = r_fromf<R>(0.0f);
  for (int e = 0; e < n * n; ++e) {
    L[e] = zero;
    Li[e] = zero;
  }
  for (int j = 0; j < d; ++j) {
    R s = S[j * n + j];
    for (int k = 0; k < j; ++k) s = r_fma(-L[j * n + k], L[j * n + k], s);
    ok = ok && r_pos(s);
    s = r_pos(s) ? s : r_fromf<R>(1.0f);
    R rs = r_rsqrt(s);
    L[j * n + j] = s * rs;
    Li[j * n + j] = rs;
    for (int i = j + 1; i < d; ++i) {
      R t = S[i * n + j];
      for (int k = 0; k < j; ++k) t = r_fma(-L[i * n + k], L[j * n + k], t);
      L[i * n + j] = t * rs;
    }
  }
  for (int j = 0; j < d; ++j)
    for (int i = j + 1; i < d; ++i) {
      R s = zero;
      for (int k = j; k < i; ++k) s = r_fma(L[i * n + k], Li[k * n + j], s);
      Li[i * n + j] = -(s * Li[i * n + i]);
    }
  return ok;
}

// ------------------------------------------------------------ matrix exponential
// Pade [6/6] approximant with scaling and squaring (||X||_1 <= 1/2 after
// scaling; truncation below 1e-16), dense runtime size d <= MAXD, one thread.

template <int MAXD>
PGV_DEV void mat_mul_rt(int d, const double* A, const double* B, double* C) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s = fma(A[i * MAXD + k], B[k * MAXD + j], s);
      C[i * MAXD + j] = s;
    }
}

// E = exp(M); all matrices stored with leading dimension MAXD.
template <int MAXD>
PGV_BIG bool expm_pade6(int d, const double* M, double* E) {
  double X[MAXD * MAXD], X2[MAXD * MAXD], X4[MAXD * MAXD], U[MAXD * MAXD], V[MAXD * MAXD];
  double nrm = 0.0;
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += fabs(M[i * MAXD + j]);
    nrm = fmax(nrm, s);
  }
  int sq = 0;
  if (nrm > 0.5) sq = (int)ceil(log2(nrm / 0.5));
  double sc = ldexp(1.0, -sq);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) X[i * MAXD + j] = M[i * MAXD + j] * sc;
  const double c1 = 1.0 / 2, c2 = 5.0 / 44, c3 = 1.0 / 66, c4 = 1.0 / 792, c5 = 1.0 / 15840,
               c6 = 1.0 / 665280;
  mat_mul_rt<MAXD>(d, X, X, X2);
  mat_mul_rt<MAXD>(d, X2, X2, X4);
  // V = I + c2 X2 + c4 X4 + c6 X2 X4 ;  U = X (c1 I + c3 X2 + c5 X4)
  mat_mul_rt<MAXD>(d, X2, X4, V);  // X6 in V
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double id = (i == j) ? 1.0 : 0.0;
      double x6 = V[i * MAXD + j];
      V[i * MAXD + j] = id + c2 * X2[i * MAXD + j] + c4 * X4[i * MAXD + j] + c6 * x6;
      U[i * MAXD + j] = c1 * id + c3 * X2[i * MAXD + j] + c5 * X4[i * MAXD + j];
    }
  mat_mul_rt<MAXD>(d, X, U, X2);  // U -> X2
  // Solve (V - U) R = (V + U) by Gaussian elimination with partial pivoting.
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double v = V[i * MAXD + j], u = X2[i * MAXD + j];
      X4[i * MAXD + j] = v - u;  // P
      E[i * MAXD + j] = v + u;   // right-hand sides
    }
  for (int c = 0; c < d; ++c) {
    int piv = c;
    double best = fabs(X4[c * MAXD + c]);
    for (int r = c + 1; r < d; ++r) {
      double v = fabs(X4[r * MAXD + c]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < d; ++j) {
        double t = X4[c * MAXD + j]; X4[c * MAXD + j] = X4[piv * MAXD + j]; X4[piv * MAXD + j] = t;
        t = E[c * MAXD + j]; E[c * MAXD + j] = E[piv * MAXD + j]; E[piv * MAXD + j] = t;
      }
    double inv = 1.0 / X4[c * MAXD + c];
    for (int r = c + 1; r < d; ++r) {
      double f = X4[r * MAXD + c] * inv;
      if (f != 0.0) {
        for (int j = c; j < d; ++j) X4[r * MAXD + j] = fma(-f, X4[c * MAXD + j], X4[r * MAXD + j]);
        for (int j = 0; j < d; ++j) E[r * MAXD + j] = fma(-f, E[c * MAXD + j], E[r * MAXD + j]);
      }
    }
  }
  for (int c = d - 1; c >= 0; --c) {
    double inv = 1.0 / X4[c * MAXD + c];
    for (int j = 0; j < d; ++j) {
      double s = E[c * MAXD + j];
      for (int k = c + 1; k < d; ++k) s = fma(-X4[c * MAXD + k], E[k * MAXD + j], s);
      E[c * MAXD + j] = s * inv;
    }
  }
  for (int s = 0; s < sq; ++s) {
    mat_mul_rt<MAXD>(d, E, E, X);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) E[i * MAXD + j] = X[i * MAXD + j];
  }
  return true;
}

// General small inverse by Gauss-Jordan (runtime size, leading dim MAXD).
template <int MAXD>
PGV_DEV bool inv_rt(int d, const double* A, double* Ai) {
  double M[MAXD * MAXD];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      M[i * MAXD + j] = A[i * MAXD + j];
      Ai[i * MAXD + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < d; ++c) {
    int piv = c;
    double best = fabs(M[c * MAXD + c]);
    for (int r = c + 1; r < d; ++r) {
      double v = fabs(M[r * MAXD + c]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != c)
      for (int j = 0; j < d; ++j) {
        double t = M[c * MAXD + j]; M[c * MAXD + j] = M[piv * MAXD + j]; M[piv * MAXD + j] = t;
        t = Ai[c * MAXD + j]; Ai[c * MAXD + j] = Ai[piv * MAXD + j]; Ai[piv * MAXD + j] = t;
      }
    double inv = 1.0 / M[c * MAXD + c];
    for (int j = 0; j < d; ++j) { M[c * MAXD + j] *= inv; Ai[c * MAXD + j] *= inv; }
    for (int r = 0; r < d; ++r) {
      if (r == c) continue;
      double f = M[r * MAXD + c];
      if (f != 0.0) {
        for (int j = 0; j < d; ++j) {
          M[r * MAXD + j] = fma(-f, M[c * MAXD + j], M[r * MAXD + j]);
          Ai[r * MAXD + j] = fma(-f, Ai[c * MAXD + j], Ai[r * MAXD + j]);
        }
      }
    }
  }
  return true;
}

// ------------------------------------------------------------------ SDF
// Node-centred grid, clamped coordinates, bilinear / trilinear interpolation.
// The grid coordinate of a query is split into an integer part (exact) and a
// fractional offset in T, so FP32 keeps sub-micro-cell resolution far from
// the map origin.

template <typename T>
PGV_DEV void clamp_axis(int base, T frac, int size, int& i0, T& f) {
  T fl = floor(frac);
  int i = base + (int)fl;
  T fr = frac - fl;
  if (i < 0) { i = 0; fr = (T)0; }
  if (i > size - 2) { i = size - 2; fr = (T)1; }
  i0 = i;
  f = fr;
}

template <typename T>
PGV_DEV T sdf2(const float* __restrict__ g, int nx, int ny, int bx, T fx, int by, T fy) {
  int ix, iy;
  T ux, uy;
  clamp_axis<T>(bx, fx, nx, ix, ux);
  clamp_axis<T>(by, fy, ny, iy, uy);
  const float* r0 = g + (size_t)iy * nx + ix;
  T v00 = (T)pgv_ldg(r0), v10 = (T)pgv_ldg(r0 + 1), v01 = (T)pgv_ldg(r0 + nx), v11 = (T)pgv_ldg(r0 + nx + 1);
  T a = v00 + ux * (v10 - v00);
  T b = v01 + ux * (v11 - v01);
  return a + uy * (b - a);
}

template <typename T>
PGV_DEV T sdf3(const float* __restrict__ g, int nx, int ny, int nz, int bx, T fx, int by, T fy, int bz, T fz) {
  int ix, iy, iz;
  T ux, uy, uz;
  clamp_axis<T>(bx, fx, nx, ix, ux);
  clamp_axis<T>(by, fy, ny, iy, uy);
  clamp_axis<T>(bz, fz, nz, iz, uz);
  const float* p = g + ((size_t)iz * ny + iy) * nx + ix;
  size_t sy = nx, sz = (size_t)nx * ny;
  T c00 = (T)pgv_ldg(p), c10 = (T)pgv_ldg(p + 1), c01 = (T)pgv_ldg(p + sy), c11 = (T)pgv_ldg(p + sy + 1);
  T d00 = (T)pgv_ldg(p + sz), d10 = (T)pgv_ldg(p + sz + 1), d01 = (T)pgv_ldg(p + sz + sy), d11 = (T)pgv_ldg(p + sz + sy + 1);
  T a0 = c00 + ux * (c10 - c00), a1 = c01 + ux * (c11 - c01);
  T b0 = d00 + ux * (d10 - d00), b1 = d01 + ux * (d11 - d01);
  T a = a0 + uy * (a1 - a0), b = b0 + uy * (b1 - b0);
  return a + uz * (b - a);
}

template <typename T>
PGV_DEV T hinge_psi(const PlanDesc& P, T h) {
  T hp = h > (T)0 ? h : (T)0;
  T w = (P.psi_form == 1) ? (T)(1.0 / (P.sigma_obs * P.sigma_obs)) : (T)P.sigma_obs;
  return w * hp * hp;
}

// Absolute grid coordinate of a world position (used by the arm, whose sphere
// centres come from forward kinematics rather than from a mean + offset).
template <typename T>
PGV_DEV void world_to_grid(const PlanDesc& P, T x, int d, int& base, T& frac) {
  T u = (x - (T)P.sdf_origin[d]) * (T)P.inv_cell;
  T fl = floor(u);
  base = (int)fl;
  frac = u - fl;
}

// Forward kinematics of the revolute chain (standard DH) and the summed
// sphere hinge cost at joint vector q.
template <typename T>
PGV_BIG T arm_cost(const PlanDesc& P, const T* q) {
  T R[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};  // 3x4 [rot | pos]
  T total = 0;
  const float* g = P.sdf;
  for (int j = 0; j < P.arm_dof; ++j) {
    T a = (T)P.dh[4 * j], al = (T)P.dh[4 * j + 1], d = (T)P.dh[4 * j + 2];
    T th = q[j] + (T)P.dh[4 * j + 3];
    T c, s;
    if (sizeof(T) == 4) { float cf, sf; sincosf((float)th, &sf, &cf); c = cf; s = sf; }
    else { double cd, sd; sincos((double)th, &sd, &cd); c = (T)cd; s = (T)sd; }
    // R <- R * Rz(th)
    for (int r = 0; r < 3; ++r) {
      T x0 = R[4 * r], x1 = R[4 * r + 1];
      R[4 * r] = x0 * c + x1 * s;
      R[4 * r + 1] = -x0 * s + x1 * c;
    }
    for (int k = P.sphere_begin[j]; k < P.sphere_begin[j + 1]; ++k) {
      T o0 = (T)P.sphere_off[3 * k], o1 = (T)P.sphere_off[3 * k + 1], o2 = (T)P.sphere_off[3 * k + 2];
      T p[3];
      for (int r = 0; r < 3; ++r) p[r] = R[4 * r] * o0 + R[4 * r + 1] * o1 + R[4 * r + 2] * o2 + R[4 * r + 3];
      int bx, by, bz;
      T fx, fy, fz;
      world_to_grid<T>(P, p[0], 0, bx, fx);
      world_to_grid<T>(P, p[1], 1, by, fy);
      world_to_grid<T>(P, p[2], 2, bz, fz);
      T sd = sdf3<T>(g, P.nx, P.ny, P.nz, bx, fx, by, fy, bz, fz);
      total += hinge_psi<T>(P, (T)P.eps + (T)P.sphere_r[k] - sd);
    }
    // R <- R * Tz(d) * Tx(a) * Rx(al)
    for (int r = 0; r < 3; ++r) R[4 * r + 3] += R[4 * r + 2] * d + R[4 * r] * a;
    T ca, sa;
    if (sizeof(T) == 4) { float cf, sf; sincosf((float)al, &sf, &cf); ca = cf; sa = sf; }
    else { double cd, sd; sincos((double)al, &sd, &cd); ca = (T)cd; sa = (T)sd; }
    for (int r = 0; r < 3; ++r) {
      T y1 = R[4 * r + 1], y2 = R[4 * r + 2];
      R[4 * r + 1] = y1 * ca + y2 * sa;
      R[4 * r + 2] = -y1 * sa + y2 * ca;
    }
  }
  return total;
}

}  // namespace pgv
