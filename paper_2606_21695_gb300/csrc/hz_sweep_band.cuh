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

// One subdomain (H warps) per block.  NY - 1 = SY P rows are cut into H bands
// of RB = SY P / H rows (a multiple of P); band B holds rows B RB .. B RB + RB,
// the last of which is also the next band's first row, computed by both warps
// with the same arithmetic (the copies agree bitwise).  Every warp runs the
// same code with B a run-time value, so the H warps share one instruction
// stream (separate unrolled bodies per band compete for the instruction
// cache).
template <int P, int SY, int H>
struct Shape {
  static constexpr int NY = SY * P + 1;
  static constexpr int RB = (NY - 1) / H;  // rows per band (+1 shared with the next band)
  static constexpr int NR = RB + 1;        // register rows per warp
  static constexpr int G = 1;              // subdomains per block
  static_assert((NY - 1) % H == 0 && RB % P == 0 && RB >= P, "bands of whole elements");
};

template <int P, int SY, bool SRC, int H>
__device__ __forceinline__ void band_body(const WarpSweepArgs& x, int l, int g, int lane, int B, float* xbuf,
                                          float4* ecg, float2* uo, double* red) {
  using S = Shape<P, SY, H>;
  constexpr int NY = S::NY;
  constexpr int NR = S::NR;
  constexpr int RB = S::RB;
  const SweepArgs& a = x.base;
  const int J0 = B * RB;
  const bool first = B == 0, last = B == H - 1;
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx;
  const int i = lane;
  const bool live = i < nlx;
  const int bar_id = 1 + g;

  // ---- x row (assembled, weights folded)
  const int ax = i % P, ex = i / P;
  const bool own_x = live && ex < a.sxe;
  const bool left_x = live && (ax == 0) && (ex >= 1);
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
  const int slot = (lane == 0) ? 0 : (lane == nlx - 1) ? 1 : 2;
  constexpr int NB = SRC ? NR : 1;
  float bet[NR];
  float bbr[NB], bbi[NB];
  float alE = 1.f, bEr = 0.f, bEi = 0.f;  // row 0 (first band) or row NY-1 (last band)
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = J0 + r;
    float be = 0.f, al = 1.f, br = 0.f, bi = 0.f;
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
    }
    const int ay = j % P, ey = j / P;
    const double wy = a.hy2 * ((ey < a.sye ? a.w[ay] : 0.0) + (ay == 0 && ey >= 1 ? a.w[P] : 0.0));
    bet[r] = (float)(be * wx_lane * wy);  // beta' = beta Wx Wy
    const float fbr = be * br, fbi = be * bi;
    if (SRC) {
      bbr[r] = fbr;
      bbi[r] = fbi;
    }
    if (j == 0 || j == NY - 1) {
      alE = al;
      bEr = SRC ? 0.f : fbr;
      bEi = SRC ? 0.f : fbi;
    } else if (slot < 2) {  // the shared row is written by both bands with the same value
      ecg[j * 2 + slot] = make_float4(al - 1.f, SRC ? 0.f : fbr, SRC ? 0.f : fbi, 0.f);
    }
  }
  __syncwarp();

  const float4* tab = static_cast<const float4*>(a.tab);
  const float sigma = (float)a.sigma, omega = (float)a.omega;
  const float cpi = (float)a.cpi, spi = (float)a.spi, scale = (float)a.two_over_nt;
  const float sy = x.sy;
  // first / last subdomain row: the one-element row is 2 x the two-element row
  // (w_0 = w_P; the missing side's halo is zero) minus the missing element's
  // diagonal term (see the cluster-of-bands kernel)
  const float kc_first = kYRows.c[P - 1][P + 1][P];
  const float kc_last = kYRows.c[P - 1][0][P];
  const int nout = last ? NR : NR - 1;  // rows this band outputs and counts
  // exchange buffer layout: [parity][band][side 0 = rows 1..P, 1 = rows RB-P..RB-1][P][32]
  auto xb = [&](int par, int band, int side, int k) -> float& {
    return xbuf[(((par * H + band) * 2 + side) * P + k) * 32 + lane];
  };
  float p[NR], pd[NR], vre[NR], vim[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { vre[r] = 0.f; vim[r] = 0.f; }

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
#pragma unroll
      for (int k = 0; k < P; ++k) {
        xb(cur, B, 0, k) = p[1 + k];
        xb(cur, B, 1, k) = p[RB - P + k];
      }
      group_barrier(bar_id, H * 32);
      float lo[P], hi[P];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        lo[k] = first ? 0.f : xb(cur, first ? 0 : B - 1, 1, k);  // rows J0-P+k
        hi[k] = last ? 0.f : xb(cur, last ? 0 : B + 1, 0, k);    // rows J0+NR+k
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int j = J0 + r;
        // (A p)_j / (Wx Wy): y taps of the row's class (element-boundary rows
        // with both elements), x part by shuffles
        const int a_r = r % P;
        const int cls = a_r == 0 ? P : a_r;
        float Y = 0.f;
#pragma unroll
        for (int t = -P; t <= P; ++t) {
          if (a_r == 0 || (a_r + t >= 0 && a_r + t <= P)) {
            const int rr = r + t;
            const float v = rr < 0 ? lo[rr + P] : rr >= NR ? hi[rr - NR] : p[rr];
            Y += kYRows.c[P - 1][cls][t + P] * v;
          }
        }
        if (r == 0 && first) Y = 2.f * Y - kc_first * p[r];
        if (r == NR - 1 && last) Y = 2.f * Y - kc_last * p[r];
        const float Ap = xr.apply(p[r], lane) + sy * Y;
        float f = pd[r] - bet[r] * Ap;
        if ((r == 0 && first) || (r == NR - 1 && last)) {
          f += (alE - 1.f) * pd[r] + bEr * tb.x + bEi * tb.y;
        } else {
          f = edge_fix(f, pd[r], &ecg[j * 2 + (slot & 1)], slot < 2, tb.x, tb.y);
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
        if (r < nout) {  // the shared row counts once
          const float2 o = uo[r * 32 + lane];
          const double dr = (double)vre[r] - (double)o.x, di = (double)vim[r] - (double)o.y;
          dn += dr * dr + di * di;
          un += (double)vre[r] * vre[r] + (double)vim[r] * vim[r];
        }
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

  // ---- outputs (a band's last row is the next band's first: written by that band)
  bool bad = false;
  if (live) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r >= nout) break;
      if (!isfinite(vre[r]) || !isfinite(vim[r])) bad = true;
      if (a.u_sub) {
        const int64_t n = (int64_t)l * nn + (int64_t)(J0 + r) * nlx + i;
        a.u_sub[2 * n] = (double)vre[r];
        a.u_sub[2 * n + 1] = (double)vim[r];
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.flags, 1);
  if (first && lane == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  const int NE = a.NE;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * NE;
  auto put = [&](int e, int t, bool has, double ur, double ui) {
    const bool iface = (e == 0) ? ifW : (e == 1) ? ifE : (e == 2) ? ifS : ifN;
    const int len = (e < 2) ? NY : nlx;
    double* dst;
    if (iface) {
      const int rn = (e == 0) ? l - 1 : (e == 1) ? l + 1 : (e == 2) ? l - a.Sx : l + a.Sx;
      dst = a.lam_out + 2 * (((int64_t)rn * 4 + (e ^ 1)) * NE + t);
    } else {
      dst = a.lam_out + 2 * (((int64_t)l * 4 + e) * NE + t);
    }
    if (iface && t < len && has) {
      const double kk = kedgeL[e * NE + t];
      const double lr = lamL[2 * (e * NE + t)], li = lamL[2 * (e * NE + t) + 1];
      dst[0] = -lr + 2.0 * kk * ui;
      dst[1] = -li - 2.0 * kk * ur;
    } else {
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  };
  if (first) {  // S edge: row 0
    for (int t = lane; t < NE; t += 32) {
      const bool mine = t == lane && live;
      put(2, t, mine, mine ? (double)vre[0] : 0.0, mine ? (double)vim[0] : 0.0);
    }
  }
  if (last) {  // N edge: row NY-1
    for (int t = lane; t < NE; t += 32) {
      const bool mine = t == lane && live;
      put(3, t, mine, mine ? (double)vre[NR - 1] : 0.0, mine ? (double)vim[NR - 1] : 0.0);
    }
  }
  if (lane == 0 || lane == nlx - 1) {  // W / E edges: this band's rows
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r >= nout) break;
      if (lane == 0) put(0, J0 + r, true, (double)vre[r], (double)vim[r]);
      if (lane == nlx - 1) put(1, J0 + r, true, (double)vre[r], (double)vim[r]);
    }
  }
  if (first && lane == 0) {
    for (int t = NY; t < NE; ++t) {
      put(0, t, false, 0.0, 0.0);
      put(1, t, false, 0.0, 0.0);
    }
  }
}

template <int P, int SY, bool SRC, int H>
__global__ void __launch_bounds__(H * 32, 7) sweep_band_kernel(const __grid_constant__ WarpSweepArgs x) {
  using S = Shape<P, SY, H>;
  constexpr int NY = S::NY;
  __shared__ float xbuf_all[S::G][2 * H * 2 * P * 32];
  __shared__ float4 ec_all[S::G][NY * 2];
  __shared__ float2 uold_all[H][S::NR * 32];
  __shared__ double red_all[S::G][2 * H];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = w / H, b = w % H;
  const int l = blockIdx.x * S::G + g;
  if (l >= x.L) return;  // the whole group leaves together (all H warps share l)
  band_body<P, SY, SRC, H>(x, l, g, lane, b, xbuf_all[g], ec_all[g], uold_all[w], red_all[g]);
}

}  // namespace band_sweep
}  // namespace hz
