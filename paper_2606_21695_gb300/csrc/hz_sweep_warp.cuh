// Warp-per-subdomain DD sweep (FP32), for subdomains of at most 32 node
// columns and NY = SY*P+1 rows: lane i owns node column i, every row of it
// in registers for the whole WaveHoltz loop (p, p-dot, v, beta'; alpha and
// beta*b only where they differ from 1 and 0: rows 0 and NY-1 in registers,
// the edge columns' other rows in a small shared table that the two edge
// lanes read).  The time step needs no barrier:
//   x part of A p: assembled 1D row, own-element neighbours gathered by P
//                  indexed shuffles plus one hand-off for the element to the
//                  left (hz_sweep_xrow.cuh), per-lane coefficients in registers;
//   y part:        assembled 1D rows whose sparsity pattern and values
//                  (in units of 4/hy^2) are fixed at compile time by row j's
//                  class (hz_gll_const.h), constant-bank operands of the FMAs.
// Same arithmetic as the block sweep (Algorithm 1, modified leapfrog and
// eq. (WaveHoltz) with the -1/(i omega) sign and 2/N_t scaling; lambda
// update -lambda - 2ik u); one subdomain per one-warp block, or per item of
// the persistent packed launch (hz_sweep_packed.cu).
#pragma once

#include <cuda_runtime.h>

#include "hz_gll_const.h"
#include "hz_internal.h"
#include "hz_sweep_xrow.cuh"

namespace hz {
namespace warp_sweep {

// Is tap t of assembled 1D row j structurally non-zero?  Row j lies in
// element j/P at position j%P; class-0 rows also touch the element below.
// ne: elements along the direction (the subdomain has ne*P+1 nodes).
__host__ __device__ constexpr bool tap(int P, int ne, int j, int t) {
  const int a = j % P, e = j / P;
  const bool own = e < ne && a + t >= 0 && a + t <= P;
  const bool below = a == 0 && e >= 1 && t <= 0 && t >= -P;
  return own || below;
}

// Sweep of subdomain l by the calling warp.  x may live in the parameter
// space (one problem per launch) or in global memory (packed launches).
// ec: per-warp shared table of the edge columns' rows; uo: per-warp shared
// stash of the previous iterate, used only when STASH and a WaveHoltz
// tolerance is set (may be null otherwise).
// RM: the interface boundary mass of a generalised transmission condition may
// be non-zero (eta != 0); without it the two terms it adds are compiled out.
// WARM: WaveHoltz starts from a.u0 instead of zero (a separate instantiation,
// so that the kernels without it compile as before).
template <int P, int SY, bool SRC, bool STASH, bool RM = true, bool WARM = false>
__device__ __forceinline__ void warp_body(const WarpSweepArgs& x, int l, float4 (*ec)[2], float2* uo) {
  constexpr int NY = SY * P + 1;
  constexpr int NB = SRC ? NY : 1;  // per-node forcing only when a source is present
  const SweepArgs& a = x.base;
  const int lane = threadIdx.x & 31;
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx;
  const int i = lane;
  const bool live = i < nlx;

  // ---- per-lane x row of the assembled stiffness (scaled by 2/hx)
  const int ax = i % P, ex = i / P;
  const bool own_x = live && ex < a.sxe;
  const bool left_x = live && (ax == 0) && (ex >= 1);
  // with beta' = beta Wx Wy the stiffness terms are divided by the lumped
  // weights: (A p)/(Wx Wy) = (Kx p)/Wx + (Ky p)/Wy, so no weight multiplies remain
  const double wx_lane = a.hx2 * ((own_x ? a.w[ax] : 0.0) + (left_x ? a.w[P] : 0.0));
  XRow<P> xr;
  xr.init(lane, nlx, a.sxe, a.Kref, a.kxs, [&](int c) {
    const int ac = c % P, ec_ = c / P;
    return a.hx2 * ((ec_ < a.sxe ? a.w[ac] : 0.0) + (ac == 0 && ec_ >= 1 ? a.w[P] : 0.0));
  });

  // ---- node coefficients and right-hand side.  alpha != 1 and (without a
  // source) b != 0 only on the subdomain edges: rows 0 and NY-1 keep them in
  // registers, the edge columns' interior rows in a shared table (alpha - 1,
  // beta b) that only the two edge lanes read.
  const int64_t nn = (int64_t)nlx * NY;
  const float* betaG = static_cast<const float*>(a.beta) + (int64_t)l * nn;
  const float* alphaG = static_cast<const float*>(a.alpha) + (int64_t)l * nn;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * a.NE;
  const int slot = (lane == 0) ? 0 : (lane == nlx - 1) ? 1 : 2;
  float bet[NY];
  float bbr[NB], bbi[NB];
  float al0 = 0.f, alN = 0.f, b0r = 0.f, b0i = 0.f, bNr = 0.f, bNi = 0.f, g0 = 0.f, gN = 0.f;
#pragma unroll
  for (int j = 0; j < NY; ++j) {
    if (!SRC && j > 0 && j < NY - 1) {
      // interior row without a source: only beta' differs from zero away from
      // the edge columns, whose entries the lanes fill in parallel below
      const double be = live ? (double)betaG[(int64_t)j * nlx + i] : 0.0;
      bet[j] = (float)(be * wx_lane * x.wyr[j]);
      continue;
    }
    double be = 0.0, al = 0.0, br = 0.0, bi = 0.0, hm = 0.0;
    if (live) {
      const int64_t n = (int64_t)j * nlx + i;
      be = (double)betaG[n];
      al = (double)alphaG[n];
      if (SRC) {
        const double shx = ((i == 0 && ifW) || (i == nlx - 1 && ifE)) ? 0.5 : 1.0;
        const double shy = ((j == 0 && ifS) || (j == NY - 1 && ifN)) ? 0.5 : 1.0;
        const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
        const double* src = a.rhs + 2 * (J * a.NXg + I);
        br = shx * shy * src[0];
        bi = shx * shy * src[1];
      }
      if (i == 0 && ifW) { br += a.wys[j] * lamL[2 * (0 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (0 * a.NE + j) + 1]; }
      if (i == nlx - 1 && ifE) { br += a.wys[j] * lamL[2 * (1 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (1 * a.NE + j) + 1]; }
      if (j == 0 && ifS) { br += a.wxs[i] * lamL[2 * (2 * a.NE + i)]; bi += a.wxs[i] * lamL[2 * (2 * a.NE + i) + 1]; }
      if (j == NY - 1 && ifN) { br += a.wxs[i] * lamL[2 * (3 * a.NE + i)]; bi += a.wxs[i] * lamL[2 * (3 * a.NE + i) + 1]; }
      // interface boundary mass (k w on each interface edge of the node)
      if (i == 0 && ifW) hm += a.wys[j] * kedgeL[0 * a.NE + j];
      if (i == nlx - 1 && ifE) hm += a.wys[j] * kedgeL[1 * a.NE + j];
      if (j == 0 && ifS) hm += a.wxs[i] * kedgeL[2 * a.NE + i];
      if (j == NY - 1 && ifN) hm += a.wxs[i] * kedgeL[3 * a.NE + i];
    }
    const float gm = (float)(-be * a.eta * hm);  // gamma = -beta w eta <c^-1 phi, phi>
    bet[j] = (float)(be * wx_lane * x.wyr[j]);  // beta' = beta Wx Wy
    const float fbr = (float)(be * br), fbi = (float)(be * bi);
    if (SRC) {
      bbr[j] = fbr;
      bbi[j] = fbi;
    }
    if (j == 0) { al0 = (float)al; b0r = SRC ? 0.f : fbr; b0i = SRC ? 0.f : fbi; g0 = gm; }
    if (j == NY - 1) { alN = (float)al; bNr = SRC ? 0.f : fbr; bNi = SRC ? 0.f : fbi; gN = gm; }
    if (j > 0 && j < NY - 1) {
      if (slot < 2) ec[j][slot] = make_float4((float)(al - 1.0), SRC ? 0.f : fbr, SRC ? 0.f : fbi, gm);
    }
  }
  if (!SRC) {
    // edge columns' interior rows, lane t taking row t of both: the same FP64
    // expressions as the per-lane rows above (lambda and the boundary mass
    // enter only on an interface edge), computed once per row rather than by
    // the two edge lanes one row after another
    for (int t = lane; t < NY - 1; t += 32) {
      if (t == 0) continue;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int cc = s == 0 ? 0 : nlx - 1;
        const bool iface = s == 0 ? ifW : ifE;
        const int64_t n = (int64_t)t * nlx + cc;
        const double be = (double)betaG[n];
        const double al = (double)alphaG[n];
        double br = 0.0, bi = 0.0, hm = 0.0;
        if (iface) {
          br += a.wys[t] * lamL[2 * (s * a.NE + t)];
          bi += a.wys[t] * lamL[2 * (s * a.NE + t) + 1];
          hm += a.wys[t] * kedgeL[s * a.NE + t];
        }
        ec[t][s] = make_float4((float)(al - 1.0), (float)(be * br), (float)(be * bi), (float)(-be * a.eta * hm));
      }
    }
  }
  __syncwarp();

  const float4* tab = static_cast<const float4*>(a.tab);
  const float sigma = (float)a.sigma, omega = (float)a.omega;
  const float cpi = (float)a.cpi, spi = (float)a.spi, scale = (float)a.two_over_nt;
  const float sy = x.sy;
  const int Nt = a.Nt, m_wh = a.m_wh;
  const bool tol = STASH && a.wh_tol > 0.0;
  const double wh_tol = a.wh_tol;
  // between WaveHoltz iterations u lives in (vre, vim); the previous iterate
  // is kept in shared memory only when a tolerance is checked
  float p[NY], pd[NY], vre[NY], vim[NY];
#pragma unroll
  for (int j = 0; j < NY; ++j) { vre[j] = 0.f; vim[j] = 0.f; }
  if (WARM && live) {  // warm start from a previous sweep's subdomain solution (a.u0)
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      const int64_t n = (int64_t)l * nn + (int64_t)j * nlx + i;
      vre[j] = (float)a.u0[2 * n];
      vim[j] = (float)a.u0[2 * n + 1];
    }
  }

  int m_done = 0;
  for (int m = 0; m < m_wh; ++m) {
    if (tol) {
#pragma unroll
      for (int j = 0; j < NY; ++j) uo[j * 32 + lane] = make_float2(vre[j], vim[j]);
    }
    {
      const float4 t0 = tab[0];
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        p[j] = vre[j];
        pd[j] = omega * (vim[j] * cpi - vre[j] * spi);  // Re{-i w u e^{-i pi/N_t}}
        vre[j] = t0.z * p[j];
        vim[j] = t0.w * pd[j];
      }
    }
    float4 tb = tab[1];
    for (int nu = 1; nu < Nt; ++nu) {
      const float4 tn = tab[nu + 1];  // prefetch (the table has N_t + 1 entries)
#pragma unroll
      for (int j = 0; j < NY; ++j) p[j] += sigma * pd[j];
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        // (A p)_j / (Wx Wy): y taps from registers (compile-time sparsity and
        // coefficients, constant-bank operands) times 4/hy^2, x part from
        // neighbour lanes
        float Y = 0.f;
#pragma unroll
        for (int t = -P; t <= P; ++t) {
          if (tap(P, SY, j, t) && j + t >= 0 && j + t < NY)
            Y += kYRows.c[P - 1][gllc::row_class(P, SY, j)][t + P] * p[j + t];
        }
        const float Ap = xr.apply(p[j], lane) + sy * Y;
        float f;
        if (j == 0) {
          f = al0 * pd[j] - bet[j] * Ap + b0r * tb.x + b0i * tb.y;
          if (RM) f += g0 * p[j];
        } else if (j == NY - 1) {
          f = alN * pd[j] - bet[j] * Ap + bNr * tb.x + bNi * tb.y;
          if (RM) f += gN * p[j];
        } else {
          f = edge_fix<RM>(pd[j] - bet[j] * Ap, pd[j], p[j], &ec[j][slot & 1], slot < 2, tb.x, tb.y);
        }
        if (SRC) f += bbr[j] * tb.x + bbi[j] * tb.y;
        pd[j] = f;
      }
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        vre[j] += tb.z * p[j];
        vim[j] += tb.w * pd[j];
      }
      tb = tn;
    }
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      vre[j] *= scale;  // u^{(m+1)} = (2/N_t) v
      vim[j] *= scale;
    }
    m_done = m + 1;
    if (tol) {
      double dn = 0.0, un = 0.0;
#pragma unroll
      for (int j = 0; j < NY; ++j) {
        const float2 o = uo[j * 32 + lane];
        const double dr = (double)vre[j] - (double)o.x, di = (double)vim[j] - (double)o.y;
        dn += dr * dr + di * di;
        un += (double)vre[j] * vre[j] + (double)vim[j] * vim[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        un += __shfl_xor_sync(0xffffffffu, un, o);
      }
      if (dn <= wh_tol * wh_tol * un) break;  // warp-uniform after the reduction
    }
  }

  // ---- outputs
  bool bad = false;
  if (live) {
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      if (!isfinite(vre[j]) || !isfinite(vim[j])) bad = true;
      if (a.u_sub) {
        const int64_t n = (int64_t)l * nn + (int64_t)j * nlx + i;
        a.u_sub[2 * n] = (double)vre[j];
        a.u_sub[2 * n + 1] = (double)vim[j];
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.flags, 1);
  if (lane == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  const int NE = a.NE;
  // S / N edges: lane i holds node (i, 0) and (i, NY-1)
  auto put = [&](int e, int t, bool has, double ur, double ui) {
    const bool iface = (e == 0) ? ifW : (e == 1) ? ifE : (e == 2) ? ifS : ifN;
    const int len = (e < 2) ? NY : nlx;
    if (iface) {
      const int r = (e == 0) ? l - 1 : (e == 1) ? l + 1 : (e == 2) ? l - a.Sx : l + a.Sx;
      double* dst = a.lam_out + 2 * (((int64_t)r * 4 + (e ^ 1)) * NE + t);
      if (t < len && has) {
        const double kk = kedgeL[e * NE + t];
        const double lr = lamL[2 * (e * NE + t)], li = lamL[2 * (e * NE + t) + 1];
        // -lambda + 2 k (eta - i zeta) u  (eta = 0, zeta = 1: -lambda - 2ik u)
        dst[0] = -lr + 2.0 * kk * (a.eta * ur + a.zeta * ui);
        dst[1] = -li + 2.0 * kk * (a.eta * ui - a.zeta * ur);
      } else {
        dst[0] = 0.0;
        dst[1] = 0.0;
      }
    } else {
      double* dst = a.lam_out + 2 * (((int64_t)l * 4 + e) * NE + t);
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  };
  for (int t = lane; t < NE; t += 32) {
    // lane t < nlx holds column t: rows 0 and NY-1 are in its registers only
    // for t == lane, which holds in the first pass (nlx <= 32)
    const bool mine = t == lane && live;
    put(2, t, mine, mine ? (double)vre[0] : 0.0, mine ? (double)vim[0] : 0.0);
    put(3, t, mine, mine ? (double)vre[NY - 1] : 0.0, mine ? (double)vim[NY - 1] : 0.0);
  }
  // W / E edges: columns 0 and nlx-1 hold every row.  They are staged in the
  // edge table (not read after the time loop) so that lane t writes row t of
  // both edges, instead of two lanes running the FP64 update row by row.
  if (slot < 2) {
#pragma unroll
    for (int j = 0; j < NY; ++j) ec[j][slot] = make_float4(vre[j], vim[j], 0.f, 0.f);
  }
  __syncwarp();
  for (int t = lane; t < NE; t += 32) {
    const bool has = t < NY;
    const float4 uw = has ? ec[t][0] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 ue = has ? ec[t][1] : make_float4(0.f, 0.f, 0.f, 0.f);
    put(0, t, has, (double)uw.x, (double)uw.y);
    put(1, t, has, (double)ue.x, (double)ue.y);
  }
}

// One subdomain (one warp) per block: 1024 subdomains spread as 6-7 blocks
// per SM over 152 SMs, instead of multi-warp blocks landing unevenly.
template <int P, int SY, bool SRC, bool RM, bool WARM = false>
__global__ void __launch_bounds__(32) sweep_warp_kernel(const __grid_constant__ WarpSweepArgs x) {
  constexpr int NY = SY * P + 1;
  __shared__ float4 ec[NY][2];
  __shared__ float2 uo[NY * 32];
  if ((int)blockIdx.x >= x.L) return;
  const int l = sweep_subdomain(x.base, blockIdx.x);
  warp_body<P, SY, SRC, true, RM, WARM>(x, l, ec, uo);
}

}  // namespace warp_sweep
}  // namespace hz
