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

#include "pgvimp_plan.h"

namespace pgv {

#ifndef PGV_DEV
#define PGV_DEV __device__ __forceinline__
#endif
// Full unrolling of the block loops only for small blocks (n <= 8).
// Large routines are inlined too: an out-of-line (__noinline__) build of the
// n = 14 trial sweep, whose thread-local arrays exceed 20 KB, returned wrong
// covariance blocks on sm_103a, while the inlined build is exact.
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

// ------------------------------------------------------------ small blocks
// Row-major n x n blocks held in thread-local arrays.

template <int n>
PGV_DEV void ld_blk(const double* p, double* X) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll (n <= 8 ? 32 : 1)
  for (int e = 0; e < n * n / 2; ++e) {
    double2 v = q[e];
    X[2 * e] = v.x;
    X[2 * e + 1] = v.y;
  }
}
template <int n>
PGV_DEV void st_blk(double* p, const double* X) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll (n <= 8 ? 32 : 1)
  for (int e = 0; e < n * n / 2; ++e) q[e] = make_double2(X[2 * e], X[2 * e + 1]);
}
template <int n>
PGV_DEV void st_blk_scaled(double* p, const double* X, double s) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll (n <= 8 ? 32 : 1)
  for (int e = 0; e < n * n / 2; ++e) q[e] = make_double2(s * X[2 * e], s * X[2 * e + 1]);
}
template <int n>
PGV_DEV void ld_vec(const double* p, double* x) {
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a) x[a] = p[a];
}
template <int n>
PGV_DEV void st_vec(double* p, const double* x) {
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a) p[a] = x[a];
}

// Y = X * Cinv with Cinv symmetric (full storage).
template <int n>
PGV_DEV void mul_nn(const double* X, const double* Y, double* Z) {
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int t = 0; t < n; ++t) s = fma(X[a * n + t], Y[t * n + c], s);
      Z[a * n + c] = s;
    }
}
// Z = X * Y^T, symmetric result assumed (lower computed, mirrored).
template <int n>
PGV_DEV void mul_nt_sym(const double* X, const double* Y, double* Z) {
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
    for (int c = 0; c <= a; ++c) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int t = 0; t < n; ++t) s = fma(X[a * n + t], Y[c * n + t], s);
      Z[a * n + c] = s;
      Z[c * n + a] = s;
    }
}
// Z = C + X^T Y, symmetric result assumed.
template <int n>
PGV_DEV void add_tn_sym(const double* C, const double* X, const double* Y, double* Z) {
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
    for (int c = 0; c <= a; ++c) {
      double s = C[a * n + c];
#pragma unroll (n <= 8 ? 32 : 1)
      for (int t = 0; t < n; ++t) s = fma(X[t * n + a], Y[t * n + c], s);
      Z[a * n + c] = s;
      Z[c * n + a] = s;
    }
}

// Accumulates pivot products as mantissa * 2^exponent so that log det needs a
// single log at the end of a sweep.
struct LogDetAcc {
  double mant;
  int expo;
  PGV_DEV void init() { mant = 1.0; expo = 0; }
  PGV_DEV void mul(double v) {
    int e;
    mant = frexp(mant * v, &e);
    expo += e;
  }
  PGV_DEV double log_value() const { return log(mant) + expo * 0.69314718055994530942; }
};

// Cholesky C = L L^T of a symmetric block, then Cinv = L^-T L^-1.
// Returns false (and leaves Cinv undefined) unless every pivot is > 0.
template <int n>
PGV_DEV bool chol_inverse(const double* C, double* Cinv, LogDetAcc& ld) {
  double L[n * n];
  double r[n];
  bool ok = true;
#pragma unroll (n <= 8 ? 32 : 1)
  for (int j = 0; j < n; ++j) {
    double s = C[j * n + j];
#pragma unroll (n <= 8 ? 32 : 1)
    for (int k = 0; k < j; ++k) s = fma(-L[j * n + k], L[j * n + k], s);
    ok = ok && (s > 0.0);
    s = ok ? s : 1.0;
    double rs = pgv_rsqrt(s);
    r[j] = rs;
    L[j * n + j] = s * rs;
    ld.mul(s);
#pragma unroll (n <= 8 ? 32 : 1)
    for (int i = j + 1; i < n; ++i) {
      double t = C[i * n + j];
#pragma unroll (n <= 8 ? 32 : 1)
      for (int k = 0; k < j; ++k) t = fma(-L[i * n + k], L[j * n + k], t);
      L[i * n + j] = t * rs;
    }
  }
  // X = L^-1 (lower), stored over L's strictly-upper-free layout in Xi
  double X[n * n];
#pragma unroll (n <= 8 ? 32 : 1)
  for (int j = 0; j < n; ++j) {
    X[j * n + j] = r[j];
#pragma unroll (n <= 8 ? 32 : 1)
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int k = j; k < i; ++k) s = fma(L[i * n + k], X[k * n + j], s);
      X[i * n + j] = -s * r[i];
    }
  }
  // Cinv = X^T X
#pragma unroll (n <= 8 ? 32 : 1)
  for (int a = 0; a < n; ++a)
#pragma unroll (n <= 8 ? 32 : 1)
    for (int c = 0; c <= a; ++c) {
      double s = 0.0;
#pragma unroll (n <= 8 ? 32 : 1)
      for (int k = a; k < n; ++k) s = fma(X[k * n + a], X[k * n + c], s);
      Cinv[a * n + c] = s;
      Cinv[c * n + a] = s;
    }
  return ok;
}

// Lower Cholesky factor and its inverse of the leading d x d block of a
// symmetric n x n block (runtime d <= n).  Returns false unless positive.
template <int n, typename T>
PGV_DEV bool chol_lead(const double* S, int d, T* L, T* Li) {
  double l[n * n], x[n * n];
  bool ok = true;
  for (int j = 0; j < d; ++j) {
    double s = S[j * n + j];
    for (int k = 0; k < j; ++k) s = fma(-l[j * n + k], l[j * n + k], s);
    ok = ok && (s > 0.0);
    s = ok ? s : 1.0;
    double rs = pgv_rsqrt(s);
    l[j * n + j] = s * rs;
    x[j * n + j] = rs;
    for (int i = j + 1; i < d; ++i) {
      double t = S[i * n + j];
      for (int k = 0; k < j; ++k) t = fma(-l[i * n + k], l[j * n + k], t);
      l[i * n + j] = t * rs;
    }
  }
  for (int j = 0; j < d; ++j)
    for (int i = j + 1; i < d; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s = fma(l[i * n + k], x[k * n + j], s);
      x[i * n + j] = -s * x[i * n + i];
    }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      L[i * n + j] = (T)(j <= i ? l[i * n + j] : 0.0);
      Li[i * n + j] = (T)(j <= i ? x[i * n + j] : 0.0);
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
