// Error bounds of the library's double-float arithmetic (df64: an unevaluated
// sum hi + lo of two floats), compiled for the host from the device header
// with floating-point contraction off, as the device build's round-to-nearest
// intrinsics are.  References are computed in long double (64-bit
// significand), far finer than the 2^-48 scale checked.  With u = 2^-24 the
// unit roundoff of float:
//   conversion from double      |err| <= 2 u^2 |v|
//   product (two-product, FMA)  |err| <= 8 u^2 |x y|
//   sum (two-sum, fast two-sum) |err| <= 4 u^2 (|x| + |y|)   (no cancellation bound)
//   fused x y + z               |err| <= 8 u^2 (|x y| + |z|)
//   1/sqrt (one Newton step)    |err| <= 16 u^2 / sqrt(v)   (the host starts from a correctly
//                                 rounded 1/sqrtf, the device from rsqrtf: the refinement is checked)
//   log det accumulator         |err| <= 16 u^2 * count in the log
//   reciprocal (one Newton step) |err| <= 8 u^2 / |v|
//   four-term dot product       |err| <= 16 u^2 sum_t |x_t y_t|   (compensated, no cancellation bound)
// Prints the largest observed error over its bound per operation, then "ok"
// when every ratio is at most 1.
#include <cmath>
#include <cstdio>
#include <random>

#include "pgvimp_dfx.cuh"

using pgv::df64;

namespace {

const long double kU2 = std::ldexp(1.0L, -48);

long double exact(df64 v) { return (long double)v.hi + (long double)v.lo; }

struct Worst {
  const char* name;
  double ratio = 0.0;
  void see(long double err, long double bound) {
    const double r = (double)(std::fabs(err) / bound);
    if (r > ratio) ratio = r;
  }
};

}  // namespace

int main() {
  std::mt19937_64 rng(20241103);
  std::uniform_real_distribution<double> mant(1.0, 2.0), expo(-20.0, 20.0), coin(0.0, 1.0);
  auto draw = [&]() {
    const double v = std::ldexp(mant(rng), (int)std::floor(expo(rng)));
    return coin(rng) < 0.5 ? -v : v;
  };
  Worst conv{"conversion"}, mul{"product"}, add{"sum"}, fma{"fused"}, rs{"rsqrt"}, ld{"logdet"}, rc{"reciprocal"},
      dot{"dot4"};
  for (int t = 0; t < 200000; ++t) {
    const double a = draw(), b = draw(), c = draw();
    const df64 x = pgv::r_from<df64>(a), y = pgv::r_from<df64>(b), z = pgv::r_from<df64>(c);
    conv.see(exact(x) - (long double)a, 2 * kU2 * std::fabs((long double)a));
    const long double X = exact(x), Y = exact(y), Z = exact(z);
    mul.see(exact(x * y) - X * Y, 8 * kU2 * std::fabs(X * Y));
    add.see(exact(x + y) - (X + Y), 4 * kU2 * (std::fabs(X) + std::fabs(Y)));
    fma.see(exact(pgv::r_fma(x, y, z)) - (X * Y + Z), 8 * kU2 * (std::fabs(X * Y) + std::fabs(Z)));
    const df64 p = pgv::r_from<df64>(std::fabs(a));
    const long double P = exact(p);
    rs.see(exact(pgv::r_rsqrt(p)) - 1.0L / std::sqrt(P), 16 * kU2 / std::sqrt(P));
    rc.see(exact(pgv::df_rcp(x)) - 1.0L / X, 8 * kU2 / std::fabs(X));
    df64 u[4], v[4];
    long double want = 0.0L, mag = 0.0L;
    for (int k = 0; k < 4; ++k) {
      u[k] = pgv::r_from<df64>(draw());
      v[k] = pgv::r_from<df64>(draw());
      want += exact(u[k]) * exact(v[k]);
      mag += std::fabs(exact(u[k]) * exact(v[k]));
    }
    dot.see(exact(pgv::df_dot4(u, v)) - want, 16 * kU2 * mag);
  }
  // dot products that nearly cancel
  for (int t = 0; t < 50000; ++t) {
    df64 u[4], v[4];
    const double a = draw(), b = draw(), d = std::ldexp(mant(rng), -(int)(20 + 20 * coin(rng)));
    u[0] = pgv::r_from<df64>(a); v[0] = pgv::r_from<df64>(b);
    u[1] = pgv::r_from<df64>(-a); v[1] = pgv::r_from<df64>(b * (1.0 + d));
    u[2] = pgv::r_from<df64>(draw() * 1e-3); v[2] = pgv::r_from<df64>(draw());
    u[3] = pgv::r_from<df64>(draw()); v[3] = pgv::r_from<df64>(draw() * 1e-3);
    long double want = 0.0L, mag = 0.0L;
    for (int k = 0; k < 4; ++k) {
      want += exact(u[k]) * exact(v[k]);
      mag += std::fabs(exact(u[k]) * exact(v[k]));
    }
    dot.see(exact(pgv::df_dot4(u, v)) - want, 16 * kU2 * mag);
  }
  // sums and fused sums that nearly cancel: y = -x (1 + d), |d| down to 2^-40
  for (int t = 0; t < 50000; ++t) {
    const double a = draw(), d = std::ldexp(mant(rng), -(int)(20 + 20 * coin(rng)));
    const df64 x = pgv::r_from<df64>(a), y = pgv::r_from<df64>(-a * (1.0 + d));
    const long double X = exact(x), Y = exact(y);
    add.see(exact(x + y) - (X + Y), 4 * kU2 * (std::fabs(X) + std::fabs(Y)));
    const df64 one = pgv::r_fromf<df64>(1.0f);
    fma.see(exact(pgv::r_fma(x, one, y)) - (X + Y), 8 * kU2 * (std::fabs(X) + std::fabs(Y)));
  }
  // log det: products of 751 pivots spanning six decades, renormalised as they go
  std::uniform_real_distribution<double> lg(-3.0, 3.0);
  for (int rep = 0; rep < 200; ++rep) {
    pgv::LogDetAcc<df64> acc;
    acc.init();
    long double want = 0.0L;
    const int count = 751;
    for (int i = 0; i < count; ++i) {
      const df64 v = pgv::r_from<df64>(std::pow(10.0, lg(rng)));
      acc.mul(v);
      want += std::log(exact(v));
    }
    ld.see((long double)acc.log_value() - want, 16 * kU2 * count + 1e-15L * std::fabs(want));
  }
  bool ok = true;
  for (const Worst* w : {&conv, &mul, &add, &fma, &rs, &ld, &rc, &dot}) {
    std::printf("%s %.3f\n", w->name, w->ratio);
    ok = ok && w->ratio <= 1.0;
  }
  std::printf("%s\n", ok ? "ok" : "FAIL");
  return ok ? 0 : 1;
}
