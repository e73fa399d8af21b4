// Register-resident FP32 sweep with H warps per subdomain (H = 2 or 4).
//
// Same arithmetic as the warp-per-subdomain kernel (hz_sweep_warp.cuh):
// lane i owns node column i (at most 32 columns), the x part of A p comes
// from neighbour lanes by shuffles (hz_sweep_xrow.cuh), the y part from rows
// held in registers.
// The NY = SY*P+1 rows are split into H bands of consecutive rows, one warp
// each, so a subdomain's state is spread over H warps: fewer registers per
// thread and H times more warps per SM to hide latency.  Each time step a
// band publishes its first and last P rows of p to a double-buffered shared
// exchange buffer, the subdomain's H warps meet at one named barrier, and each
// band reads the P halo rows above and below it (the same single-barrier
// double-buffer argument as for the block kernel, restricted to the group).
#pragma once

#include <cuda_runtime.h>

#include "hz_internal.h"
#include "hz_sweep_warp.cuh"

namespace hz {
namespace band_sweep {


__device__ __forceinline__ void group_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// One subdomain (H warps) per block.
template <int P, int SY, int H>
struct Shape {
  static constexpr int NY = SY * P + 1;
  static constexpr int RB = (NY + H - 1) / H;  // rows per band (the last band may be shorter)
  static constexpr int G = 1;                   // subdomains per block
};

template <int P, int SY, bool SRC, int H, int B, bool WARM>
__device__ __forceinline__ void band_body(const WarpSweepArgs& x, int l, int g, int lane, float* xbuf, float4* ecg,
                                          float2* uo, double* red) {
  using S = Shape<P, SY, H>;
  constexpr int NY = S::NY;
  constexpr int J0 = B * S::RB;
  constexpr int J1 = (B + 1) * S::RB < NY ? (B + 1) * S::RB : NY;
  constexpr int NR = J1 - J0;
  static_assert(NR >= P, "every band must hold at least P rows");
  constexpr bool HAS_LO = B > 0, HAS_HI = B < H - 1;
  const SweepArgs& a = x.base;
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx;
  const int i = lane;
  const bool live = i < nlx;
  const int bar_id = 1 + g;

  // ---- per-lane x row (scaled by 2/hx)
  const int ax = i % P, ex = i / P;
  const bool own_x = live && ex < a.sxe;
  const bool left_x = live && (ax == 0) && (ex >= 1);
  // with beta' = beta Wx Wy the stiffness terms are divided by the lumped
  // weights: (A p)/(Wx Wy) = (Kx p)/Wx + (Ky p)/Wy
  const double wx_lane = a.hx2 * ((own_x ? a.w[ax] : 0.0) + (left_x ? a.w[P] : 0.0));
  XRow<P> xr;
  xr.init(lane, nlx, a.sxe, a.Kref, a.kxs, [&](int c) {
    const int ac = c % P, ec_ = c / P;
    return a.hx2 * ((ec_ < a.sxe ? a.w[ac] : 0.0) + (ac == 0 && ec_ >= 1 ? a.w[P] : 0.0));
  });

  // ---- node data of the band's rows (edge data as in the warp kernel)
  const int64_t nn = (int64_t)nlx * NY;
  const float* betaG = static_cast<const float*>(a.beta) + (int64_t)l * nn;
  const float* alphaG = static_cast<const float*>(a.alpha) + (int64_t)l * nn;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * a.NE;
  const int slot = (lane == 0) ? 0 : (lane == nlx - 1) ? 1 : 2;
  constexpr int NB = SRC ? NR : 1;
  float bet[NR];
  float bbr[NB], bbi[NB];
  float alE = 0.f, bEr = 0.f, bEi = 0.f, gE = 0.f;  // row 0 (band 0) or row NY-1 (last band)
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = J0 + r;
    float be = 0.f, al = 0.f, br = 0.f, bi = 0.f;
    double hm = 0.0;
    if (live) {
      const int64_t n = (int64_t)j * nlx + i;
      be = betaG[n];
      al = alphaG[n];
      if (SRC) {
        const float shx = ((i == 0 && ifW) || (i == nlx - 1 && ifE)) ? 0.5f : 1.f;
        const float shy = ((j == 0 && ifS) || (j == NY - 1 && ifN)) ? 0.5f : 1.f;
        const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
        const double* src = a.rhs + 2 * (J * a.NXg + I);
        br = shx * shy * (float)src[0];
        bi = shx * shy * (float)src[1];
      }
      if (i == 0 && ifW) { br += (float)(a.wys[j] * lamL[2 * (0 * a.NE + j)]); bi += (float)(a.wys[j] * lamL[2 * (0 * a.NE + j) + 1]); }
      if (i == nlx - 1 && ifE) { br += (float)(a.wys[j] * lamL[2 * (1 * a.NE + j)]); bi += (float)(a.wys[j] * lamL[2 * (1 * a.NE + j) + 1]); }
      if (j == 0 && ifS) { br += (float)(a.wxs[i] * lamL[2 * (2 * a.NE + i)]); bi += (float)(a.wxs[i] * lamL[2 * (2 * a.NE + i) + 1]); }
      if (j == NY - 1 && ifN) { br += (float)(a.wxs[i] * lamL[2 * (3 * a.NE + i)]); bi += (float)(a.wxs[i] * lamL[2 * (3 * a.NE + i) + 1]); }
      // interface boundary mass (k w on each interface edge of the node)
      if (i == 0 && ifW) hm += a.wys[j] * kedgeL[0 * a.NE + j];
      if (i == nlx - 1 && ifE) hm += a.wys[j] * kedgeL[1 * a.NE + j];
      if (j == 0 && ifS) hm += a.wxs[i] * kedgeL[2 * a.NE + i];
      if (j == NY - 1 && ifN) hm += a.wxs[i] * kedgeL[3 * a.NE + i];
    }
    const float gm = (float)(-(double)be * a.eta * hm);  // gamma = -beta w eta <c^-1 phi, phi>
    bet[r] = (float)(be * wx_lane * x.wyr[j]);  // beta' = beta Wx Wy
    const float fbr = be * br, fbi = be * bi;
    if (SRC) {
      bbr[r] = fbr;
      bbi[r] = fbi;
    }
    if (j == 0 || j == NY - 1) { alE = al; bEr = SRC ? 0.f : fbr; bEi = SRC ? 0.f : fbi; gE = gm; }
    if (j > 0 && j < NY - 1) {
      if (slot < 2) ecg[j * 2 + slot] = make_float4(al - 1.f, SRC ? 0.f : fbr, SRC ? 0.f : fbi, gm);
    }
  }
  __syncwarp();

  const float4* tab = static_cast<const float4*>(a.tab);
  const float sigma = (float)a.sigma, omega = (float)a.omega;
  const float cpi = (float)a.cpi, spi = (float)a.spi, scale = (float)a.two_over_nt;
  const float sy = x.sy;
  // exchange buffer layout: [parity][band][side 0 = first P rows, 1 = last P rows][P][32]
  auto xb = [&](int par, int band, int side, int k) -> float& {
    return xbuf[(((par * H + band) * 2 + side) * P + k) * 32 + lane];
  };
  float p[NR], pd[NR], vre[NR], vim[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { vre[r] = 0.f; vim[r] = 0.f; }
  if (WARM && live) {  // warm start from a previous sweep's subdomain solution (a.u0, this band's rows)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int64_t n = (int64_t)l * nn + (int64_t)(J0 + r) * nlx + i;
      vre[r] = (float)a.u0[2 * n];
      vim[r] = (float)a.u0[2 * n + 1];
    }
  }

  int m_done = 0;
  // buffer parity runs on across WaveHoltz iterations: consecutive time steps
  // always alternate buffers (N_t - 1 may be odd), which the single barrier
  // per step relies on
  int cur = 0;
  for (int m = 0; m < a.m_wh; ++m) {
    if (a.wh_tol > 0.0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) uo[r * 32 + lane] = make_float2(vre[r], vim[r]);
    }
    {
      const float4 t0 = tab[0];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        p[r] = vre[r];
        pd[r] = omega * (vim[r] * cpi - vre[r] * spi);  // Re{-i w u e^{-i pi/N_t}}
        vre[r] = t0.z * p[r];
        vim[r] = t0.w * pd[r];
      }
    }
    float4 tb = tab[1];
    for (int nu = 1; nu < a.Nt; ++nu) {
      const float4 tn = tab[nu + 1];  // prefetch (the table has N_t + 1 entries)
#pragma unroll
      for (int r = 0; r < NR; ++r) p[r] += sigma * pd[r];
      if (HAS_LO) {
#pragma unroll
        for (int k = 0; k < P; ++k) xb(cur, B, 0, k) = p[k];
      }
      if (HAS_HI) {
#pragma unroll
        for (int k = 0; k < P; ++k) xb(cur, B, 1, k) = p[NR - P + k];
      }
      group_barrier(bar_id, H * 32);
      float lo[P], hi[P];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        lo[k] = HAS_LO ? xb(cur, B - 1, 1, k) : 0.f;  // rows J0-P+k
        hi[k] = HAS_HI ? xb(cur, B + 1, 0, k) : 0.f;  // rows J1+k
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int j = J0 + r;
        // (A p)_j / (Wx Wy): y taps (registers and halo rows, compile-time
        // coefficients times 4/hy^2), x part by shuffles
        float Y = 0.f;
#pragma unroll
        for (int t = -P; t <= P; ++t) {
          const int jj = j + t;
          if (warp_sweep::tap(P, SY, j, t) && jj >= 0 && jj < NY) {
            const float v = (jj < J0) ? lo[jj - (J0 - P)] : (jj >= J1) ? hi[jj - J1] : p[jj - J0];
            Y += kYRows.c[P - 1][gllc::row_class(P, SY, j)][t + P] * v;
          }
        }
        const float Ap = xr.apply(p[r], lane) + sy * Y;
        float f;
        if (j == 0 || j == NY - 1) {
          f = alE * pd[r] - bet[r] * Ap + bEr * tb.x + bEi * tb.y + gE * p[r];
        } else {
          f = edge_fix(pd[r] - bet[r] * Ap, pd[r], p[r], &ecg[j * 2 + (slot & 1)], slot < 2, tb.x, tb.y);
        }
        if (SRC) f += bbr[r] * tb.x + bbi[r] * tb.y;
        pd[r] = f;
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        vre[r] += tb.z * p[r];
        vim[r] += tb.w * pd[r];
      }
      tb = tn;
      cur ^= 1;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      vre[r] *= scale;  // u^{(m+1)} = (2/N_t) v
      vim[r] *= scale;
    }
    m_done = m + 1;
    if (a.wh_tol > 0.0) {
      double dn = 0.0, un = 0.0;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float2 o = uo[r * 32 + lane];
        const double dr = (double)vre[r] - (double)o.x, di = (double)vim[r] - (double)o.y;
        dn += dr * dr + di * di;
        un += (double)vre[r] * vre[r] + (double)vim[r] * vim[r];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        un += __shfl_xor_sync(0xffffffffu, un, o);
      }
      if (lane == 0) { red[2 * B] = dn; red[2 * B + 1] = un; }
      group_barrier(bar_id, H * 32);
      double D = 0.0, U = 0.0;
#pragma unroll
      for (int bb = 0; bb < H; ++bb) { D += red[2 * bb]; U += red[2 * bb + 1]; }  // same order in every band
      group_barrier(bar_id, H * 32);  // red[] read by all bands before it can be rewritten
      if (D <= a.wh_tol * a.wh_tol * U) break;
    }
  }

  // ---- outputs
  bool bad = false;
  if (live) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (!isfinite(vre[r]) || !isfinite(vim[r])) bad = true;
      if (a.u_sub) {
        const int64_t n = (int64_t)l * nn + (int64_t)(J0 + r) * nlx + i;
        a.u_sub[2 * n] = (double)vre[r];
        a.u_sub[2 * n + 1] = (double)vim[r];
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.flags, 1);
  if (B == 0 && lane == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  const int NE = a.NE;
  auto put = [&](int e, int t, bool has, double ur, double ui) {
    const bool iface = (e == 0) ? ifW : (e == 1) ? ifE : (e == 2) ? ifS : ifN;
    const int len = (e < 2) ? NY : nlx;
    double* dst;
    if (iface) {
      const int r = (e == 0) ? l - 1 : (e == 1) ? l + 1 : (e == 2) ? l - a.Sx : l + a.Sx;
      dst = a.lam_out + 2 * (((int64_t)r * 4 + (e ^ 1)) * NE + t);
    } else {
      dst = a.lam_out + 2 * (((int64_t)l * 4 + e) * NE + t);
    }
    if (iface && t < len && has) {
      const double kk = kedgeL[e * NE + t];
      const double lr = lamL[2 * (e * NE + t)], li = lamL[2 * (e * NE + t) + 1];
      // -lambda + 2 k (eta - i zeta) u  (eta = 0, zeta = 1: -lambda - 2ik u)
      dst[0] = -lr + 2.0 * kk * (a.eta * ur + a.zeta * ui);
      dst[1] = -li + 2.0 * kk * (a.eta * ui - a.zeta * ur);
    } else {
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  };
  if (B == 0) {  // S edge: row 0
    for (int t = lane; t < NE; t += 32) {
      const bool mine = t == lane && live;
      put(2, t, mine, mine ? (double)vre[0] : 0.0, mine ? (double)vim[0] : 0.0);
    }
  }
  if (B == H - 1) {  // N edge: row NY-1
    for (int t = lane; t < NE; t += 32) {
      const bool mine = t == lane && live;
      put(3, t, mine, mine ? (double)vre[NR - 1] : 0.0, mine ? (double)vim[NR - 1] : 0.0);
    }
  }
  if (lane == 0 || lane == nlx - 1) {  // W / E edges: this band's rows
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (lane == 0) put(0, J0 + r, true, (double)vre[r], (double)vim[r]);
      if (lane == nlx - 1) put(1, J0 + r, true, (double)vre[r], (double)vim[r]);
    }
  }
  if (B == 0 && lane == 0) {
    for (int t = NY; t < NE; ++t) {
      put(0, t, false, 0.0, 0.0);
      put(1, t, false, 0.0, 0.0);
    }
  }
}

template <int P, int SY, bool SRC, int H, bool WARM = false>
__global__ void __launch_bounds__(H * 32, 7) sweep_band_kernel(const __grid_constant__ WarpSweepArgs x) {
  using S = Shape<P, SY, H>;
  constexpr int NY = S::NY;
  __shared__ float xbuf_all[S::G][2 * H * 2 * P * 32];
  __shared__ float4 ec_all[S::G][NY * 2];
  __shared__ float2 uold_all[H][S::RB * 32];
  __shared__ double red_all[S::G][2 * H];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = w / H, b = w % H;
  const int k = blockIdx.x * S::G + g;
  if (k >= x.L) return;  // the whole group leaves together (all H warps share l)
  const int l = sweep_subdomain(x.base, k);
  float* xbuf = xbuf_all[g];
  float4* ecg = ec_all[g];
  float2* uo = uold_all[w];
  double* red = red_all[g];
  if (b == 0) band_body<P, SY, SRC, H, 0, WARM>(x, l, g, lane, xbuf, ecg, uo, red);
  else if (b == 1) band_body<P, SY, SRC, H, (H > 1 ? 1 : 0), WARM>(x, l, g, lane, xbuf, ecg, uo, red);
  else if (b == 2) band_body<P, SY, SRC, H, (H > 2 ? 2 : 0), WARM>(x, l, g, lane, xbuf, ecg, uo, red);
  else band_body<P, SY, SRC, H, (H > 3 ? 3 : 0), WARM>(x, l, g, lane, xbuf, ecg, uo, red);
}

}  // namespace band_sweep
}  // namespace hz
