// Host-side discretisation set-up (Sec. 4 and 5): GLL nodes and weights,
// the reference 1D stiffness, lumped 1D weights, and the largest eigenvalue
// of the 1D subdomain operator used by the time-step rule.
#include <cmath>
#include <string>
#include <vector>

#include "hz_gll_const.h"
#include "hz_internal.h"

namespace hz {
namespace {

std::vector<double> lumped(int n_el, int P, double h, const std::vector<double>& w) {
  std::vector<double> W(n_el * P + 1, 0.0);
  for (int e = 0; e < n_el; ++e)
    for (int a = 0; a <= P; ++a) W[e * P + a] += w[a] * h / 2.0;
  return W;
}

// Largest eigenvalue of a dense symmetric matrix (cyclic Jacobi rotations).
double max_eig_sym(std::vector<double> A, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        tot += A[p * n + q] * A[p * n + q];
        if (p != q) off += A[p * n + q] * A[p * n + q];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[p * n + p], aqq = A[q * n + q];
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
      }
  }
  double m = A[0];
  for (int k = 1; k < n; ++k) m = std::fmax(m, A[k * n + k]);
  return m;
}

}  // namespace

hz_status build_geom(double x0, double x1, double y0, double y1, int nx, int ny, int P, int snx, int sny, Geom* g) {
  if (!(x1 > x0) || !(y1 > y0) || !std::isfinite(x0) || !std::isfinite(x1) || !std::isfinite(y0) ||
      !std::isfinite(y1))
    return fail(HZ_ERR_INVALID_ARG, "empty or non-finite box");
  if (P < 1 || P > kMaxP) return fail(HZ_ERR_INVALID_ARG, "degree must be in 1..7");
  if (nx < 1 || ny < 1 || snx < 1 || sny < 1) return fail(HZ_ERR_INVALID_ARG, "element counts must be >= 1");
  if (nx % snx || ny % sny) return fail(HZ_ERR_INVALID_ARG, "subdomain size must divide the element counts");
  if ((int64_t)nx * P + 1 > (1 << 20) || (int64_t)ny * P + 1 > (1 << 20))
    return fail(HZ_ERR_INVALID_ARG, "mesh too large");
  g->x0 = x0; g->x1 = x1; g->y0 = y0; g->y1 = y1;
  g->nx = nx; g->ny = ny; g->P = P; g->snx = snx; g->sny = sny;
  g->hx = (x1 - x0) / nx;
  g->hy = (y1 - y0) / ny;
  g->Sx = nx / snx;
  g->Sy = ny / sny;
  g->L = g->Sx * g->Sy;
  g->NXg = nx * P + 1;
  g->NYg = ny * P + 1;
  g->n = (int64_t)g->NXg * g->NYg;
  g->nlx = snx * P + 1;
  g->nly = sny * P + 1;
  g->NE = g->nlx > g->nly ? g->nlx : g->nly;
  // the same construction the kernels' compile-time tables come from
  const gllc::Gll G = gllc::make_gll(P);
  g->xi.assign(G.x, G.x + P + 1);
  g->w.assign(G.w, G.w + P + 1);
  g->Kref.assign(G.K, G.K + (P + 1) * (P + 1));
  g->Wxg = lumped(nx, P, g->hx, g->w);
  g->Wyg = lumped(ny, P, g->hy, g->w);
  g->Wxs = lumped(snx, P, g->hx, g->w);
  g->Wys = lumped(sny, P, g->hy, g->w);
  return HZ_OK;
}

double max_eig_1d(const Geom& g, int n_el, double h) {
  const int P = g.P;
  const int n = n_el * P + 1;
  std::vector<double> K((size_t)n * n, 0.0);
  for (int e = 0; e < n_el; ++e)
    for (int a = 0; a <= P; ++a)
      for (int b = 0; b <= P; ++b) K[(size_t)(e * P + a) * n + e * P + b] += (2.0 / h) * g.Kref[a * (P + 1) + b];
  const std::vector<double> W = lumped(n_el, P, h, g.w);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) K[(size_t)p * n + q] /= std::sqrt(W[p] * W[q]);
  return max_eig_sym(K, n);
}

}  // namespace hz
