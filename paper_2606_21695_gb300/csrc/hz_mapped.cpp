// Geometry of meshes of general convex quadrilaterals (HZ_NODE_COORDS).
//
// Sec. 4 of the paper allows convex quadrilateral elements.  Each element is
// the isoparametric image of the reference square [-1, 1]^2 through its
// (P+1)^2 GLL nodes: x(xi, eta) and y(xi, eta) are the degree-P Lagrange
// interpolants of the given node coordinates.  With the collocated GLL rule
// the Galerkin stiffness (grad phi_j, grad phi_i) becomes, per element,
//   u_xi  = sum_c D[a][c] u(c, b),   u_eta = sum_c D[b][c] u(a, c)
//   F1    = w_a w_b (G11 u_xi + G12 u_eta),   F2 = w_a w_b (G12 u_xi + G22 u_eta)
//   (A u)(a', b') += sum_a D[a][a'] F1(a, b') + sum_b D[b][b'] F2(a', b)
// with J = x_xi y_eta - x_eta y_xi and
//   G11 = (x_eta^2 + y_eta^2) / J,  G12 = -(x_xi x_eta + y_xi y_eta) / J,
//   G22 = (x_xi^2 + y_xi^2) / J;
// the lumped mass at a node is the sum of w_a w_b J over its elements and the
// boundary integrals carry the arc-length factor |(x_xi, y_xi)| (edges along
// xi) or |(x_eta, y_eta)| (edges along eta).  Everything here is host FP64,
// computed once when the coordinates are set; the kernels read the results.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hz_problem.h"

namespace hz {
namespace {

// D[q (P+1) + a] = l_a'(xi_q) for the Lagrange basis on the nodes x
// (barycentric weights lam_a = 1 / prod_{b != a} (x_a - x_b)).
std::vector<double> lagrange_diff(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> lam(n, 1.0), D((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a) {
    double p = 1.0;
    for (int b = 0; b < n; ++b)
      if (b != a) p *= x[a] - x[b];
    lam[a] = 1.0 / p;
  }
  for (int q = 0; q < n; ++q) {
    double diag = 0.0;
    for (int a = 0; a < n; ++a) {
      if (a == q) continue;
      const double v = (lam[a] / lam[q]) / (x[q] - x[a]);
      D[(size_t)q * n + a] = v;
      diag -= v;
    }
    D[(size_t)q * n + q] = diag;
  }
  return D;
}

// Largest eigenvalue of W_e^-1/2 A_e W_e^-1/2 for one element (metric g3 =
// (P+1)^2 x 3 weighted entries, jw = w_a w_b J), by power iteration on the
// assembled dense element matrix; a Gershgorin row-sum bound first, so that
// elements that cannot exceed `best` are skipped.
double element_lambda(int P, const std::vector<double>& D, const double* g3, const double* jw, double best) {
  const int m = P + 1, n = m * m;
  std::vector<double> A((size_t)n * n, 0.0), u(n), uxi(n), ueta(n), F1(n), F2(n);
  for (int k = 0; k < n; ++k) {  // column k = A e_k
    std::fill(u.begin(), u.end(), 0.0);
    u[k] = 1.0;
    for (int b = 0; b < m; ++b)
      for (int q = 0; q < m; ++q) {
        double sx = 0.0, se = 0.0;
        for (int c = 0; c < m; ++c) {
          sx += D[q * m + c] * u[b * m + c];
          se += D[b * m + c] * u[c * m + q];
        }
        uxi[b * m + q] = sx;
        ueta[b * m + q] = se;
      }
    for (int e = 0; e < n; ++e) {
      F1[e] = g3[3 * e] * uxi[e] + g3[3 * e + 1] * ueta[e];
      F2[e] = g3[3 * e + 1] * uxi[e] + g3[3 * e + 2] * ueta[e];
    }
    for (int b = 0; b < m; ++b)
      for (int a = 0; a < m; ++a) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += D[q * m + a] * F1[b * m + q] + D[q * m + b] * F2[q * m + a];
        A[(size_t)(b * m + a) * n + k] = s;
      }
  }
  std::vector<double> sc(n);
  for (int e = 0; e < n; ++e) sc[e] = 1.0 / std::sqrt(jw[e]);
  double gers = 0.0;
  for (int r = 0; r < n; ++r) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += std::fabs(A[(size_t)r * n + k] * sc[r] * sc[k]);
    gers = std::max(gers, s);
  }
  if (gers <= best) return 0.0;
  std::vector<double> v(n), w(n);
  for (int k = 0; k < n; ++k) v[k] = ((k % 2) ? -1.0 : 1.0) * (1.0 + 0.1 * std::sin(1.7 * k + 0.3));
  double rq = 0.0;
  for (int it = 0; it < 80; ++it) {
    double nv = 0.0;
    for (int k = 0; k < n; ++k) nv += v[k] * v[k];
    nv = std::sqrt(nv);
    for (int k = 0; k < n; ++k) v[k] /= nv;
    rq = 0.0;
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[(size_t)r * n + k] * sc[r] * sc[k] * v[k];
      w[r] = s;
      rq += v[r] * s;
    }
    v.swap(w);
  }
  return rq;
}

}  // namespace

hz_status set_node_coords(Problem& pr, const double* xy) {
  const Geom& g = pr.g;
  const int P = g.P, m = P + 1, n2 = m * m;
  if (g.sub_nodes() > 1024)
    return fail(HZ_ERR_UNSUPPORTED, "mapped meshes need subdomains of at most 1024 nodes");
  const std::vector<double> D = lagrange_diff(g.xi);
  const int64_t NX = g.NXg, NY = g.NYg;
  const int64_t nel = (int64_t)g.nx * g.ny;
  std::vector<double> geog((size_t)nel * n2 * 3), jwg((size_t)nel * n2);
  std::vector<double> Wg((size_t)g.n, 0.0), bw((size_t)(2 * NX + 2 * NY), 0.0);
  const int64_t nsub = (int64_t)g.L * g.sub_nodes();
  std::vector<double> Ws((size_t)nsub, 0.0), Es((size_t)g.L * 4 * g.NE, 0.0);
  std::vector<double> geos((size_t)nel * n2 * 3);
  std::vector<double> X(n2), Y(n2);
  const int64_t oS = 0, oE = NX, oN = NX + NY, oW = 2 * NX + NY;
  for (int ey = 0; ey < g.ny; ++ey)
    for (int ex = 0; ex < g.nx; ++ex) {
      for (int b = 0; b < m; ++b)
        for (int a = 0; a < m; ++a) {
          const int64_t k = ((int64_t)ey * P + b) * NX + (int64_t)ex * P + a;
          X[b * m + a] = xy[2 * k];
          Y[b * m + a] = xy[2 * k + 1];
        }
      const int64_t e = (int64_t)ey * g.nx + ex;
      const int sx = ex / g.snx, sy = ey / g.sny, lx = ex % g.snx, ly = ey % g.sny;
      const int l = sy * g.Sx + sx;
      const int64_t es = ((int64_t)l * g.sny + ly) * g.snx + lx;  // element index in subdomain-major order
      for (int b = 0; b < m; ++b)
        for (int a = 0; a < m; ++a) {
          double x_xi = 0, y_xi = 0, x_eta = 0, y_eta = 0;
          for (int c = 0; c < m; ++c) {
            x_xi += D[a * m + c] * X[b * m + c];
            y_xi += D[a * m + c] * Y[b * m + c];
            x_eta += D[b * m + c] * X[c * m + a];
            y_eta += D[b * m + c] * Y[c * m + a];
          }
          const double J = x_xi * y_eta - x_eta * y_xi;
          if (!(J > 0.0) || !std::isfinite(J))
            return fail(HZ_ERR_INVALID_ARG, "node coordinates give a non-positive Jacobian in element (" +
                                                std::to_string(ex) + ", " + std::to_string(ey) + ")");
          const double ww = g.w[a] * g.w[b];
          const double G11 = (x_eta * x_eta + y_eta * y_eta) / J;
          const double G12 = -(x_xi * x_eta + y_xi * y_eta) / J;
          const double G22 = (x_xi * x_xi + y_xi * y_xi) / J;
          const int loc = b * m + a;
          double* gg = &geog[((size_t)e * n2 + loc) * 3];
          gg[0] = ww * G11;
          gg[1] = ww * G12;
          gg[2] = ww * G22;
          double* gs = &geos[((size_t)es * n2 + loc) * 3];
          gs[0] = gg[0];
          gs[1] = gg[1];
          gs[2] = gg[2];
          jwg[(size_t)e * n2 + loc] = ww * J;
          const int64_t I = (int64_t)ex * P + a, Jn = (int64_t)ey * P + b;
          Wg[(size_t)(Jn * NX + I)] += ww * J;
          const int i = lx * P + a, j = ly * P + b;
          Ws[(size_t)((int64_t)l * g.sub_nodes() + (int64_t)j * g.nlx + i)] += ww * J;
          const double s_xi = std::sqrt(x_xi * x_xi + y_xi * y_xi);
          const double s_eta = std::sqrt(x_eta * x_eta + y_eta * y_eta);
          // outer boundary edges (S, E, N, W order of HZ_BOUNDARY)
          if (b == 0 && ey == 0) bw[(size_t)(oS + I)] += g.w[a] * s_xi;
          if (b == P && ey == g.ny - 1) bw[(size_t)(oN + I)] += g.w[a] * s_xi;
          if (a == 0 && ex == 0) bw[(size_t)(oW + Jn)] += g.w[b] * s_eta;
          if (a == P && ex == g.nx - 1) bw[(size_t)(oE + Jn)] += g.w[b] * s_eta;
          // subdomain edges (W, E, S, N slots of the lambda layout)
          double* E = &Es[(size_t)l * 4 * g.NE];
          if (a == 0 && lx == 0) E[0 * g.NE + j] += g.w[b] * s_eta;
          if (a == P && lx == g.snx - 1) E[1 * g.NE + j] += g.w[b] * s_eta;
          if (b == 0 && ly == 0) E[2 * g.NE + i] += g.w[a] * s_xi;
          if (b == P && ly == g.sny - 1) E[3 * g.NE + i] += g.w[a] * s_xi;
        }
    }
  // outer-boundary weight per node (corners: both edges)
  std::vector<double> Hw((size_t)g.n, 0.0);
  for (int64_t I = 0; I < NX; ++I) {
    Hw[(size_t)I] += bw[(size_t)(oS + I)];
    Hw[(size_t)((NY - 1) * NX + I)] += bw[(size_t)(oN + I)];
  }
  for (int64_t J = 0; J < NY; ++J) {
    Hw[(size_t)(J * NX)] += bw[(size_t)(oW + J)];
    Hw[(size_t)(J * NX + NX - 1)] += bw[(size_t)(oE + J)];
  }
  // lumped-mass share of each subdomain copy
  std::vector<double> share((size_t)nsub);
  for (int l = 0; l < g.L; ++l) {
    const int sx = l % g.Sx, sy = l / g.Sx;
    for (int j = 0; j < g.nly; ++j)
      for (int i = 0; i < g.nlx; ++i) {
        const int64_t I = (int64_t)sx * g.snx * P + i, J = (int64_t)sy * g.sny * P + j;
        const size_t k = (size_t)((int64_t)l * g.sub_nodes() + (int64_t)j * g.nlx + i);
        share[k] = Ws[k] / Wg[(size_t)(J * NX + I)];
      }
  }
  // element bound of lambda_max(W^-1 A)
  double mu = 0.0;
  for (int64_t e = 0; e < nel; ++e)
    mu = std::max(mu, element_lambda(P, D, &geog[(size_t)e * n2 * 3], &jwg[(size_t)e * n2], mu));
  // upload
  HZ_CUDA(cudaSetDevice(pr.device));
  auto up = [](DevBuf& dst, const void* src, size_t bytes) -> hz_status {
    HZ_TRY(dst.ensure(bytes));
    HZ_CUDA(cudaMemcpy(dst.ptr, src, bytes, cudaMemcpyHostToDevice));
    return HZ_OK;
  };
  std::vector<float> geos32(geos.size());
  for (size_t k = 0; k < geos.size(); ++k) geos32[k] = (float)geos[k];
  HZ_TRY(up(pr.mgeo64, geos.data(), geos.size() * sizeof(double)));
  HZ_TRY(up(pr.mgeo32, geos32.data(), geos32.size() * sizeof(float)));
  HZ_TRY(up(pr.mWs, Ws.data(), Ws.size() * sizeof(double)));
  HZ_TRY(up(pr.mEs, Es.data(), Es.size() * sizeof(double)));
  HZ_TRY(up(pr.mshare, share.data(), share.size() * sizeof(double)));
  HZ_TRY(up(pr.mgeog, geog.data(), geog.size() * sizeof(double)));
  HZ_TRY(up(pr.mWg, Wg.data(), Wg.size() * sizeof(double)));
  HZ_TRY(up(pr.mHw, Hw.data(), Hw.size() * sizeof(double)));
  HZ_TRY(up(pr.mbw, bw.data(), bw.size() * sizeof(double)));
  HZ_TRY(pr.mflux.ensure((size_t)nel * n2 * 4 * sizeof(double)));
  HZ_UPLOADS_DONE();
  pr.mapped_D = D;
  pr.mapped_mu = mu;
  pr.mapped = true;
  return HZ_OK;
}

}  // namespace hz
