// Compile-time Gauss-Lobatto-Legendre data (Sec. 4) for degrees 1..kMaxP, and
// the assembled 1D stiffness rows the register-resident sweeps apply in y.
//
// A subdomain node row j (ne elements, ne*P+1 nodes) falls in one of P+2
// classes; its assembled row, divided by the row's lumped weight, is a fixed
// set of numbers in units of (2/h)/(h/2) = 4/h^2.  The kernels read them from
// a __constant__ table whose initializer is evaluated by the compiler, so the
// coefficients are constant-bank operands shared by every problem, and only
// the scalar 4/h^2 is per problem.  The host builds a mesh's nodes, weights
// and reference stiffness with the same functions (hz_geom.cpp).
#pragma once

#include "hz_internal.h"

#ifdef __CUDACC__
#define HZ_HD __host__ __device__
#else
#define HZ_HD
#endif

namespace hz {
namespace gllc {

constexpr double kPi = 3.14159265358979323846;

// cos x for |x| <= pi by its Taylor series (40 terms: far below double
// rounding there); only used for the starting points of Newton's method.
HZ_HD constexpr double cos_series(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 40; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}

HZ_HD constexpr double cabs(double v) { return v < 0 ? -v : v; }

// Legendre L_P(x) and L_{P-1}(x) by the three-term recurrence.
struct LegPair {
  double lp, lpm1;
};
HZ_HD constexpr LegPair legendre(int P, double x) {
  double l0 = 1.0, l1 = x;
  if (P == 0) return {1.0, 0.0};
  for (int k = 1; k < P; ++k) {
    const double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    l0 = l1;
    l1 = l2;
  }
  return {l1, l0};
}

struct Gll {
  double x[kMaxP + 1] = {};
  double w[kMaxP + 1] = {};
  double K[(kMaxP + 1) * (kMaxP + 1)] = {};  // int_{-1}^{1} l_a' l_b', row a
};

// Nodes: +-1 and the roots of L_P' (Newton on L_P' from the Chebyshev-Lobatto
// points, L_P'' from the Legendre equation); weights 2/(P(P+1) L_P(x_k)^2);
// D[q][a] = l_a'(x_q) in closed form; K = D^T diag(w) D (exact: the integrand
// has degree 2P-2 <= 2P-1).
HZ_HD constexpr Gll make_gll(int P) {
  Gll g{};
  g.x[0] = -1.0;
  g.x[P] = 1.0;
  for (int k = 1; k < P; ++k) {
    double z = -cos_series(kPi * k / P);
    for (int it = 0; it < 100; ++it) {
      const LegPair L = legendre(P, z);
      const double d1 = P * (L.lpm1 - z * L.lp) / (1.0 - z * z);
      const double d2 = (2.0 * z * d1 - P * (P + 1.0) * L.lp) / (1.0 - z * z);
      const double dz = d1 / d2;
      z -= dz;
      if (cabs(dz) < 1e-16) break;
    }
    g.x[k] = z;
  }
  double LPv[kMaxP + 1] = {};
  for (int k = 0; k <= P; ++k) {
    LPv[k] = legendre(P, g.x[k]).lp;
    g.w[k] = 2.0 / (P * (P + 1.0) * LPv[k] * LPv[k]);
  }
  double D[(kMaxP + 1) * (kMaxP + 1)] = {};
  for (int q = 0; q <= P; ++q)
    for (int a = 0; a <= P; ++a)
      if (q != a) D[q * (P + 1) + a] = LPv[q] / (LPv[a] * (g.x[q] - g.x[a]));
  D[0] = -P * (P + 1.0) / 4.0;
  D[P * (P + 1) + P] = P * (P + 1.0) / 4.0;
  for (int a = 0; a <= P; ++a)
    for (int b = 0; b <= P; ++b) {
      double s = 0.0;
      for (int q = 0; q <= P; ++q) s += g.w[q] * D[q * (P + 1) + a] * D[q * (P + 1) + b];
      g.K[a * (P + 1) + b] = s;
    }
  return g;
}

// Row classes: 0 first node (own element only); a = 1..P-1 interior node a
// of an element; P element boundary inside the subdomain (own element and the
// one below); P+1 last node (element below only).
HZ_HD constexpr int row_class(int P, int ne, int j) {
  const int a = j % P, e = j / P;
  if (j == 0) return 0;
  if (e >= ne) return P + 1;
  return a == 0 ? P : a;
}

struct YRows {
  float c[kMaxP][kMaxP + 2][2 * kMaxP + 1] = {};  // [P-1][class][t+P], t = -P..P
};

HZ_HD constexpr YRows make_yrows() {
  YRows y{};
  for (int P = 1; P <= kMaxP; ++P) {
    const Gll g = make_gll(P);
    for (int cls = 0; cls <= P + 1; ++cls) {
      const int a = (cls == P || cls == P + 1) ? 0 : cls;
      const bool own = cls != P + 1;
      const bool below = cls == P || cls == P + 1;
      const double wsum = (own ? g.w[a] : 0.0) + (below ? g.w[P] : 0.0);
      for (int t = -P; t <= P; ++t) {
        double v = 0.0;
        if (own && a + t >= 0 && a + t <= P) v += g.K[a * (P + 1) + a + t];
        if (below && t <= 0) v += g.K[P * (P + 1) + P + t];
        y.c[P - 1][cls][t + P] = (float)(v / wsum);
      }
    }
  }
  return y;
}

}  // namespace gllc

#ifdef __CUDACC__
// One copy per translation unit (each is its own device module).
static __constant__ gllc::YRows kYRows = gllc::make_yrows();
#endif

}  // namespace hz
