// Cluster of warp bands: FP32 DD sweep (Algorithm 1) for subdomains wider
// than 32 node columns, degree dividing 32 (P = 1, 2, 4), a fixed WaveHoltz
// count or a per-subdomain WaveHoltz tolerance (a cluster-wide reduction of
// the update norm after every iteration).
//
// A subdomain of nlx x NY nodes is cut into column bands of 32 nodes, one CTA
// of a thread-block cluster each (CN = ceil(nlx / 32) CTAs); inside a CTA the
// NY = 16 W + 1 rows are cut into W row bands, one warp each: band B holds
// rows 16 B .. 16 B + 16 (17 rows; the last is also the next band's first,
// computed by both warps with identical arithmetic, so the copies agree
// bitwise).  Every warp runs the same code with B a run-time value -- one
// instruction stream per SM instead of one per band (separate fully unrolled
// bodies per band overflow the instruction cache).  Lane l of a warp owns
// node column 32 q + l of its CTA q and the warp's rows of it in registers
// for the whole WaveHoltz loop, as in the one-warp kernel (hz_sweep_warp.cuh):
// y taps from registers with compile-time coefficients (element-boundary
// rows use the two-element row; the subdomain's first and last rows are
// corrected to their one-element rows), x part by the element gather and
// hand-off inside the band (hz_sweep_xrow.cuh, XRowBand).  Per time step a
// warp publishes
//   - its rows 1..P and 16-P..15 to a shared exchange buffer (the warps
//     below and above read them as y halo), and
//   - the band's edge columns to the neighbouring CTAs through distributed
//     shared memory: lanes 32-P .. 31 into the right neighbour's left halo,
//     lane 0 into the left neighbour's right halo,
// then one cluster barrier (release / acquire) makes all of it visible; the
// buffers are double-buffered by step parity, so one barrier per step is
// enough (a buffer is rewritten two steps later, after every thread passed
// the barrier that follows its last read).
//
// Arithmetic as in the other sweeps: modified leapfrog, eq. (WaveHoltz) with
// the -1/(i omega) sign and 2/N_t scaling, lambda update -lambda - 2ik u;
// beta' = beta Wx Wy with the lumped weights folded into the stencil.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hz_gll_const.h"
#include "hz_internal.h"
#include "hz_sweep_warp.cuh"
#include "hz_sweep_xrow.cuh"

namespace hz {
namespace cband {
namespace {

namespace cg = cooperative_groups;

// RB rows per band (16, or 8 for twice the warps at half the registers)
template <int P, int SY, int RB_>
struct Shape {
  static constexpr int NY = SY * P + 1;
  static constexpr int RB = RB_;                // rows per band (+1 shared with the next band)
  static constexpr int NR = RB + 1;             // register rows per warp
  static constexpr int W = (NY - 1) / RB;       // row bands (warps per CTA)
  static_assert((NY - 1) % RB == 0 && RB % P == 0, "bands of RB rows on element boundaries");
  static_assert(32 % P == 0, "column bands must start on element boundaries");
  static_assert(W >= 2 && W <= 32, "2 to 32 row bands");
};

template <int P, int SY, int RB>
struct Smem {
  using S = Shape<P, SY, RB>;
  float xb[2][S::W][2][P][32];  // row halos: [parity][band][first / last P rows][k][lane]
  float hl[2][S::NY][P];        // left column halo: columns c0-P .. c0-1
  float hr[2][S::NY];           // right column halo: column c0+32
  float4 ecol[S::NY];           // this CTA's edge column (W or E): alpha-1, beta b
  double red[S::W][2];          // tolerance mode: per-warp partial norms
  double part[2];               // and this CTA's, read by the cluster
  int stop;
};

template <int P, int SY, int RB, bool SRC, bool TOL>
__device__ __forceinline__ void band_body(const SweepArgs& a, int l, int q, int CN, int B, int lane,
                                          Smem<P, SY, RB>& sm, Smem<P, SY, RB>* right, Smem<P, SY, RB>* left,
                                          cg::cluster_group& cluster) {
  using S = Shape<P, SY, RB>;
  constexpr int NY = S::NY;
  constexpr int NR = S::NR;
  constexpr int W = S::W;
  const int J0 = S::RB * B;
  const bool first = B == 0, last = B == W - 1;  // the band holds row 0 / row NY-1
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx;
  const int c0 = 32 * q;
  const int c = c0 + lane;
  const bool live = c < nlx;

  // ---- x row (band form) and weights
  auto wx = [&](int cc) {
    const int ac = cc % P, ec_ = cc / P;
    return a.hx2 * ((ec_ < a.sxe ? a.w[ac] : 0.0) + (ac == 0 && ec_ >= 1 ? a.w[P] : 0.0));
  };
  const double wx_lane = live ? wx(c) : 0.0;
  XRowBand<P> xr;
  xr.init(lane, c0, nlx, a.sxe, a.Kref, a.kxs, wx);

  // ---- node data of the band's rows
  const int64_t nn = (int64_t)nlx * NY;
  const float* betaG = static_cast<const float*>(a.beta) + (int64_t)l * nn;
  const float* alphaG = static_cast<const float*>(a.alpha) + (int64_t)l * nn;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  const bool edge = live && (c == 0 || c == nlx - 1);
  const double* kedgeL = a.kedge + (int64_t)l * 4 * a.NE;
  constexpr int NB = SRC ? NR : 1;
  float bet[NR];
  float bbr[NB], bbi[NB];
  float alE = 1.f, bEr = 0.f, bEi = 0.f, gE = 0.f;  // row 0 (first band) or row NY-1 (last band)
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = J0 + r;
    double be = 0.0, al = 1.0, br = 0.0, bi = 0.0, hm = 0.0;
    if (live) {
      const int64_t n = (int64_t)j * nlx + c;
      be = (double)betaG[n];
      al = (double)alphaG[n];
      if (SRC) {
        const double shx = ((c == 0 && ifW) || (c == nlx - 1 && ifE)) ? 0.5 : 1.0;
        const double shy = ((j == 0 && ifS) || (j == NY - 1 && ifN)) ? 0.5 : 1.0;
        const int64_t I = (int64_t)sxi * a.snxP + c, J = (int64_t)syi * a.snyP + j;
        const double* src = a.rhs + 2 * (J * a.NXg + I);
        br = shx * shy * src[0];
        bi = shx * shy * src[1];
      }
      if (c == 0 && ifW) { br += a.wys[j] * lamL[2 * (0 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (0 * a.NE + j) + 1]; }
      if (c == nlx - 1 && ifE) { br += a.wys[j] * lamL[2 * (1 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (1 * a.NE + j) + 1]; }
      if (j == 0 && ifS) { br += a.wxs[c] * lamL[2 * (2 * a.NE + c)]; bi += a.wxs[c] * lamL[2 * (2 * a.NE + c) + 1]; }
      if (j == NY - 1 && ifN) { br += a.wxs[c] * lamL[2 * (3 * a.NE + c)]; bi += a.wxs[c] * lamL[2 * (3 * a.NE + c) + 1]; }
      // interface boundary mass (k w on each interface edge of the node)
      if (c == 0 && ifW) hm += a.wys[j] * kedgeL[0 * a.NE + j];
      if (c == nlx - 1 && ifE) hm += a.wys[j] * kedgeL[1 * a.NE + j];
      if (j == 0 && ifS) hm += a.wxs[c] * kedgeL[2 * a.NE + c];
      if (j == NY - 1 && ifN) hm += a.wxs[c] * kedgeL[3 * a.NE + c];
    }
    const float gm = (float)(-be * a.eta * hm);  // gamma = -beta w eta <c^-1 phi, phi>
    const int ay = j % P, ey = j / P;
    const double wy = a.hy2 * ((ey < a.sye ? a.w[ay] : 0.0) + (ay == 0 && ey >= 1 ? a.w[P] : 0.0));
    bet[r] = (float)(be * wx_lane * wy);  // beta' = beta Wx Wy
    const float fbr = (float)(be * br), fbi = (float)(be * bi);
    if (SRC) {
      bbr[r] = fbr;
      bbi[r] = fbi;
    }
    if (j == 0 || j == NY - 1) {
      alE = (float)al;
      bEr = SRC ? 0.f : fbr;
      bEi = SRC ? 0.f : fbi;
      gE = gm;
    } else if (edge) {
      sm.ecol[j] = make_float4((float)(al - 1.0), SRC ? 0.f : fbr, SRC ? 0.f : fbi, gm);
    }
  }
  __syncwarp();

  const float4* tab = static_cast<const float4*>(a.tab);
  const float sigma = (float)a.sigma, omega = (float)a.omega;
  const float cpi = (float)a.cpi, spi = (float)a.spi, scale = (float)a.two_over_nt;
  const float sy = (float)(4.0 / ((2.0 * a.hy2) * (2.0 * a.hy2)));  // 4 / hy^2
  // first / last subdomain row: the one-element row is 2 x the two-element row
  // (w_0 = w_P; the missing side's halo is zero) minus the missing element's
  // diagonal term: Kref[P][P] / w_0 for the first row, Kref[0][0] / w_P for the last
  const float kc_first = kYRows.c[P - 1][P + 1][P];  // last-row class, t = 0: Kref[P][P] / w_P
  const float kc_last = kYRows.c[P - 1][0][P];       // first-row class, t = 0: Kref[0][0] / w_0
  const int Nt = a.Nt, m_wh = a.m_wh;
  const bool push_right = q < CN - 1 && lane >= 32 - P;
  const bool push_left = q > 0 && lane == 0;
  float p[NR], pd[NR], vre[NR], vim[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { vre[r] = 0.f; vim[r] = 0.f; }

  // buffer parity runs on across WaveHoltz iterations (see the block kernel)
  int cur = 0;
  int m_done = 0;
  const int nout = last ? NR : NR - 1;  // row 16 of a band is the next band's row 0
  float ore[TOL ? NR : 1], oim[TOL ? NR : 1];  // previous iterate (tolerance mode)
  for (int m = 0; m < m_wh; ++m) {
    if (TOL) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        ore[r] = vre[r];
        oim[r] = vim[r];
      }
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
    for (int nu = 1; nu < Nt; ++nu) {
      const float4 tn = tab[nu + 1];  // prefetch (the table has N_t + 1 entries)
#pragma unroll
      for (int r = 0; r < NR; ++r) p[r] += sigma * pd[r];
      // y halos for the neighbouring warps: rows 1..P (to the band below), 16-P..15 (above)
#pragma unroll
      for (int k = 0; k < P; ++k) {
        sm.xb[cur][B][0][k][lane] = p[1 + k];
        sm.xb[cur][B][1][k][lane] = p[S::RB - P + k];
      }
      if (push_right) {
#pragma unroll
        for (int r = 0; r < NR; ++r) right->hl[cur][J0 + r][lane - (32 - P)] = p[r];
      }
      if (push_left) {
#pragma unroll
        for (int r = 0; r < NR; ++r) left->hr[cur][J0 + r] = p[r];
      }
      cluster.sync();
      float lo[P], hi[P];
#pragma unroll
      for (int k = 0; k < P; ++k) {
        lo[k] = first ? 0.f : sm.xb[cur][first ? 0 : B - 1][1][k][lane];  // rows J0-P+k
        hi[k] = last ? 0.f : sm.xb[cur][last ? 0 : B + 1][0][k][lane];    // rows J0+17+k
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int j = J0 + r;
        // (A p)_j / (Wx Wy): y taps of the row's class (compile-time: r % P,
        // element-boundary rows with both elements), x part in the band plus
        // the column halos
        const int a_r = r % P;
        const int cls = a_r == 0 ? P : a_r;
        float Y = 0.f;
#pragma unroll
        for (int t = -P; t <= P; ++t) {
          const bool tp = a_r == 0 ? true : (a_r + t >= 0 && a_r + t <= P);
          if (tp) {
            const int rr = r + t;
            const float v = rr < 0 ? lo[rr + P] : rr >= NR ? hi[rr - NR] : p[rr];
            Y += kYRows.c[P - 1][cls][t + P] * v;
          }
        }
        if (r == 0) {
          if (first) Y = 2.f * Y - kc_first * p[r];
        }
        if (r == NR - 1) {
          if (last) Y = 2.f * Y - kc_last * p[r];
        }
        float hL[P];
#pragma unroll
        for (int b = 0; b < P; ++b) hL[b] = sm.hl[cur][j][b];
        const float Ap = xr.apply(p[r], lane, sm.hr[cur][j], hL) + sy * Y;
        float f = pd[r] - bet[r] * Ap;
        const bool srow = (r == 0 && first) || (r == NR - 1 && last);
        if (srow) {
          f += (alE - 1.f) * pd[r] + bEr * tb.x + bEi * tb.y + gE * p[r];
        } else {
          f = edge_fix(f, pd[r], p[r], &sm.ecol[j], edge, tb.x, tb.y);
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
    if (TOL) {
      // per-subdomain stop: ||u^{m+1} - u^m|| <= wh_tol ||u^{m+1}|| over the
      // whole subdomain; partial sums per warp, per CTA, then every CTA adds
      // the cluster's partials in the same order, so all take the same decision
      double dn = 0.0, un = 0.0;
      if (live) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nout) break;
          const double dr = (double)vre[r] - ore[r], di = (double)vim[r] - oim[r];
          dn += dr * dr + di * di;
          un += (double)vre[r] * vre[r] + (double)vim[r] * vim[r];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        un += __shfl_xor_sync(0xffffffffu, un, o);
      }
      if (lane == 0) {
        sm.red[B][0] = dn;
        sm.red[B][1] = un;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double D = 0.0, U = 0.0;
        for (int w = 0; w < W; ++w) {
          D += sm.red[w][0];
          U += sm.red[w][1];
        }
        sm.part[0] = D;
        sm.part[1] = U;
      }
      cluster.sync();
      if (threadIdx.x == 0) {
        double D = 0.0, U = 0.0;
        for (int r = 0; r < CN; ++r) {
          const double* pr = cluster.map_shared_rank(sm.part, r);
          D += pr[0];
          U += pr[1];
        }
        sm.stop = (D <= a.wh_tol * a.wh_tol * U) ? 1 : 0;
      }
      cluster.sync();  // remote reads of part[] done, stop visible to the CTA
      if (sm.stop) break;
    }
  }

  // ---- outputs (row 16 of a band is the next band's row 0: written once, by that band)
  bool bad = false;
  if (live) {
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r >= nout) break;
      if (!isfinite(vre[r]) || !isfinite(vim[r])) bad = true;
      if (a.u_sub) {
        const int64_t n = (int64_t)l * nn + (int64_t)(J0 + r) * nlx + c;
        a.u_sub[2 * n] = (double)vre[r];
        a.u_sub[2 * n + 1] = (double)vim[r];
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.flags, 1);
  if (q == 0 && first && lane == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  const int NE = a.NE;
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
      // -lambda + 2 k (eta - i zeta) u  (eta = 0, zeta = 1: -lambda - 2ik u)
      dst[0] = -lr + 2.0 * kk * (a.eta * ur + a.zeta * ui);
      dst[1] = -li + 2.0 * kk * (a.eta * ui - a.zeta * ur);
    } else {
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  };
  if (first && live) put(2, c, true, (double)vre[0], (double)vim[0]);                  // S edge: row 0
  if (last && live) put(3, c, true, (double)vre[NR - 1], (double)vim[NR - 1]);         // N edge: row NY-1
  if (edge) {  // W / E edges: this band's rows
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nout) put(c == 0 ? 0 : 1, J0 + r, true, (double)vre[r], (double)vim[r]);
  }
  if (q == 0) {  // padding entries of the edge slots (NE = max(nlx, NY))
    if (first)
      for (int t = nlx + lane; t < NE; t += 32) put(2, t, false, 0.0, 0.0);
    if (last)
      for (int t = nlx + lane; t < NE; t += 32) put(3, t, false, 0.0, 0.0);
    if (first && lane == 0)
      for (int t = NY; t < NE; ++t) {
        put(0, t, false, 0.0, 0.0);
        put(1, t, false, 0.0, 0.0);
      }
  }
}

template <int P, int SY, int RB, bool SRC, bool TOL>
__global__ void __launch_bounds__(Shape<P, SY, RB>::W * 32) sweep_cband_kernel(const __grid_constant__ SweepArgs a) {
  __shared__ Smem<P, SY, RB> sm;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int CN = (int)cluster.num_blocks();
  const int l = sweep_subdomain(a, blockIdx.x / CN);  // the whole cluster shares one subdomain
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // zero the halos (read before any neighbour writes at the domain edges)
  {
    float* z = reinterpret_cast<float*>(&sm);
    for (int k = threadIdx.x; k < (int)(sizeof(sm) / sizeof(float)); k += blockDim.x) z[k] = 0.f;
  }
  Smem<P, SY, RB>* right = q < CN - 1 ? cluster.map_shared_rank(&sm, q + 1) : nullptr;
  Smem<P, SY, RB>* left = q > 0 ? cluster.map_shared_rank(&sm, q - 1) : nullptr;
  cluster.sync();  // every CTA's buffers zeroed before any neighbour pushes into them
  band_body<P, SY, RB, SRC, TOL>(a, l, q, CN, w, lane, sm, right, left, cluster);
  cluster.sync();  // no CTA leaves while a neighbour may still touch its shared memory
}

template <int P, int SY, int RB>
hz_status launch(const SweepArgs& a, int L, cudaStream_t st) {
  using S = Shape<P, SY, RB>;
  const int CN = (a.nlx + 31) / 32;
  if (CN < 2 || CN > 8) return HZ_ERR_UNSUPPORTED;
  const bool tol = a.wh_tol > 0.0;
  auto kern = a.rhs ? (tol ? sweep_cband_kernel<P, SY, RB, true, true> : sweep_cband_kernel<P, SY, RB, true, false>)
                    : (tol ? sweep_cband_kernel<P, SY, RB, false, true> : sweep_cband_kernel<P, SY, RB, false, false>);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(L * CN));
  cfg.blockDim = dim3((unsigned)(S::W * 32));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)CN;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    (void)cudaGetLastError();
    return HZ_ERR_UNSUPPORTED;
  }
  HZ_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  note_launch();
  return HZ_OK;
}

template <int P, int SY>
hz_status launch_rb(const SweepArgs& a, int L, cudaStream_t st) {
  if (a.ty_force == 8) return launch<P, SY, 8>(a, L, st);
  return launch<P, SY, 16>(a, L, st);
}

}  // namespace
}  // namespace cband

hz_status launch_sweep_cband(int P, const SweepArgs& a, int L, cudaStream_t st) {
  if (a.round_mode != 0) return HZ_ERR_UNSUPPORTED;  // FP32 only
  if (a.nlx <= 32) return HZ_ERR_UNSUPPORTED;
  // rows per warp band: 16 (a.ty_force != 8) or 8
  const int sy = (a.nly - 1) / P;
  if (P == 4 && sy == 32) return cband::launch_rb<4, 32>(a, L, st);
  if (P == 4 && sy == 16) return cband::launch_rb<4, 16>(a, L, st);
  if (P == 2 && sy == 32) return cband::launch_rb<2, 32>(a, L, st);
  if (P == 2 && sy == 16) return cband::launch_rb<2, 16>(a, L, st);
  return HZ_ERR_UNSUPPORTED;
}

}  // namespace hz
