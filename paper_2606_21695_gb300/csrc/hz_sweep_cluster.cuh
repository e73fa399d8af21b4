// Cluster DD sweep (FP32 or FP64) for subdomains too large for one thread block.
//
// A subdomain is split into CN column bands; band q is solved by CTA q of a
// thread-block cluster (one cluster per subdomain, all subdomains in one
// launch).  Inside a band the layout is that of the block sweep: thread =
// node column x strip of P*TY rows, state in registers, p published each
// time step to a double-buffered shared tile with a zero halo.  The halo
// columns that belong to the neighbouring bands are *pushed*: the threads
// owning a band's first / last P columns also store their p into the left /
// right neighbour's tile through distributed shared memory, and one cluster
// barrier (release/acquire at cluster scope) per time step makes the local
// and remote stores visible -- the same single-barrier double-buffer
// argument as in one block, extended to the cluster.
//
// The kernel is compiled for FP32 (hz_sweep_cluster_f32.cu) and FP64
// (hz_sweep_cluster_f64.cu, the plain-FP64 path for subdomains too large
// for one block).
//
// Arithmetic is that of the block sweep (Algorithm 1; modified leapfrog;
// eq. (WaveHoltz) with the -1/(i omega) sign and 2/N_t scaling; lambda
// update -lambda - 2ik u).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "hz_internal.h"

namespace cg = cooperative_groups;

namespace hz {
namespace cluster_sweep {
namespace {

// 4-wide table entries / edge-column records in the working precision
template <typename Real>
struct alignas(4 * sizeof(Real)) Vec4 {
  Real x, y, z, w;
};
template <typename Real>
__device__ __forceinline__ Real kref(const SweepArgs& a, int k);
template <>
__device__ __forceinline__ float kref<float>(const SweepArgs& a, int k) { return a.Kref32[k]; }
template <>
__device__ __forceinline__ double kref<double>(const SweepArgs& a, int k) { return a.Kref[k]; }

// Threads per CTA at most: 512 with 2P rows per thread (TY = 2, up to 128
// registers), 256 with 4P rows (TY = 4, up to 255 registers).
template <int TY>
struct ClusterBlock {
  static constexpr int kMaxThreads = TY >= 4 ? 256 : 512;
};

// SRC: the sweep carries a source (every node forced); without it, alpha != 1
// and the forcing live only on the subdomain's edges, kept out of the
// per-thread registers: the first and last node rows in six registers, the
// edge columns' other rows in a shared table read by the edge threads only.
template <typename Real, int P, int TY, int CN, bool SRC>
__global__ void __launch_bounds__(ClusterBlock<TY>::kMaxThreads) sweep_cluster_kernel(const __grid_constant__ SweepArgs a,
                                                                                   int BW) {
  constexpr int RY = P * TY;
  constexpr int NK = 2 * P + 1;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);

  const int q = (int)cluster.block_rank();
  const int l = sweep_subdomain(a, blockIdx.x / CN);
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx, nly = a.nly;
  const int i0 = q * BW;
  const int bw = min(BW, nlx - i0);
  const int t = threadIdx.x;
  const int il = t % BW;
  const int s = t / BW;
  const bool active = (il < bw) && (s < a.NS);
  const int ile = (il < bw) ? il : 0;
  const int se = (s < a.NS) ? s : 0;  // inactive threads read valid cells, never write
  const int i = i0 + ile;
  const int j0 = se * RY;
  const int colsP = BW + 2 * P;
  const int rowsP = a.NS * RY + P + 1;
  const int PS = rowsP * colsP;
  Real* buf0 = sm;
  Real* buf1 = sm + PS;
  Real* stash = sm + 2 * PS;  // previous iterate (tolerance mode), (re, im) per node
  // edge-column table (no source): row j of this band's W (slot 0) / E (slot 1) column,
  // at a 16-byte aligned offset after the tiles and the stash
  Vec4<Real>* ecol = reinterpret_cast<Vec4<Real>*>(sm + ((2 * PS + 2 * nly * BW + 3) & ~3));

  for (int k = t; k < 2 * PS; k += blockDim.x) sm[k] = Real(0);
  Real* left0 = q > 0 ? cluster.map_shared_rank(buf0, q - 1) : nullptr;
  Real* left1 = q > 0 ? cluster.map_shared_rank(buf1, q - 1) : nullptr;
  Real* right0 = q < CN - 1 ? cluster.map_shared_rank(buf0, q + 1) : nullptr;
  Real* right1 = q < CN - 1 ? cluster.map_shared_rank(buf1, q + 1) : nullptr;
  const bool push_left = active && q > 0 && il < P;
  const bool push_right = active && q < CN - 1 && il >= bw - P;

  // ---- per-thread x row of the assembled stiffness (scaled by 2/hx), weights
  const int ax = i % P, ex = i / P;
  const bool own_x = ex < a.sxe;
  const bool left_x = (ax == 0) && (ex >= 1);
  Real kx[NK];
#pragma unroll
  for (int tt = 0; tt < NK; ++tt) {
    const int off = tt - P;
    double v = 0.0;
    const int b = ax + off;
    if (own_x && b >= 0 && b <= P) v += a.Kref[ax * (P + 1) + b];
    if (left_x && off <= 0) v += a.Kref[P * (P + 1) + (off + P)];
    kx[tt] = (Real)(v * a.kxs);
  }
  const Real wxy = (Real)(a.kys * a.hx2 * ((own_x ? a.w[ax] : 0.0) + (left_x ? a.w[P] : 0.0)));
  Real wy[RY];
  Real eok[TY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int ay = r % P;
    const int ey = (j0 + r) / P;
    const bool own_y = ey < a.sye;
    const bool below_y = (ay == 0) && (ey >= 1);
    wy[r] = (Real)(a.hy2 * ((own_y ? a.w[ay] : 0.0) + (below_y ? a.w[P] : 0.0)));
  }
#pragma unroll
  for (int qq = 0; qq < TY; ++qq) eok[qq] = (se * TY + qq < a.sye) ? Real(1) : Real(0);
  const Real bok = (se > 0) ? Real(1) : Real(0);

  // ---- node coefficients and right-hand side
  const int64_t nn = (int64_t)nlx * nly;
  const Real* betaG = static_cast<const Real*>(a.beta) + (int64_t)l * nn;
  const Real* alphaG = static_cast<const Real*>(a.alpha) + (int64_t)l * nn;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  constexpr int NR = SRC ? RY : 1;
  const double* kedgeE = a.kedge + (int64_t)l * 4 * a.NE;
  Real bet[RY], alp[NR], bbr[NR], bbi[NR], gam[NR];
  // no source: first / last node row of the subdomain (all columns), and the edge columns
  Real al0 = 1, b0r = 0, b0i = 0, g0 = 0, alN = 1, bNr = 0, bNi = 0, gN = 0;
  const int slot = (i == 0) ? 0 : (i == nlx - 1) ? 1 : 2;
  const bool edge_col = active && slot < 2;
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = j0 + r;
    const bool live = active && (j < nly);
    double be = 0.0, al = 0.0, br = 0.0, bi = 0.0, hm = 0.0;
    if (live) {
      const int64_t n = (int64_t)j * nlx + i;
      be = (double)betaG[n];
      al = (double)alphaG[n];
      if (SRC) {
        const double shx = ((i == 0 && ifW) || (i == nlx - 1 && ifE)) ? 0.5 : 1.0;
        const double shy = ((j == 0 && ifS) || (j == nly - 1 && ifN)) ? 0.5 : 1.0;
        const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
        const double* src = a.rhs + 2 * (J * a.NXg + I);
        br = shx * shy * src[0];
        bi = shx * shy * src[1];
      }
      if (i == 0 && ifW) { br += a.wys[j] * lamL[2 * (0 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (0 * a.NE + j) + 1]; }
      if (i == nlx - 1 && ifE) { br += a.wys[j] * lamL[2 * (1 * a.NE + j)]; bi += a.wys[j] * lamL[2 * (1 * a.NE + j) + 1]; }
      if (j == 0 && ifS) { br += a.wxs[i] * lamL[2 * (2 * a.NE + i)]; bi += a.wxs[i] * lamL[2 * (2 * a.NE + i) + 1]; }
      if (j == nly - 1 && ifN) { br += a.wxs[i] * lamL[2 * (3 * a.NE + i)]; bi += a.wxs[i] * lamL[2 * (3 * a.NE + i) + 1]; }
      // interface boundary mass (k w on each interface edge of the node)
      if (i == 0 && ifW) hm += a.wys[j] * kedgeE[0 * a.NE + j];
      if (i == nlx - 1 && ifE) hm += a.wys[j] * kedgeE[1 * a.NE + j];
      if (j == 0 && ifS) hm += a.wxs[i] * kedgeE[2 * a.NE + i];
      if (j == nly - 1 && ifN) hm += a.wxs[i] * kedgeE[3 * a.NE + i];
    }
    const Real gm = (Real)(-be * a.eta * hm);  // gamma = -beta w eta <c^-1 phi, phi>
    bet[r] = (Real)be;
    if (SRC) {
      alp[r] = (Real)al;
      bbr[r] = (Real)(be * br);
      bbi[r] = (Real)(be * bi);
      gam[r] = gm;
    } else if (live) {
      if (j == 0) { al0 = (Real)al; b0r = (Real)(be * br); b0i = (Real)(be * bi); g0 = gm; }
      if (j == nly - 1) { alN = (Real)al; bNr = (Real)(be * br); bNi = (Real)(be * bi); gN = gm; }
      if (j > 0 && j < nly - 1 && slot < 2)
        ecol[j * 2 + slot] = Vec4<Real>{(Real)(al - 1.0), (Real)(be * br), (Real)(be * bi), gm};
    }
  }

  const Vec4<Real>* tab = static_cast<const Vec4<Real>*>(a.tab);
  const Real sigma = (Real)a.sigma, omega = (Real)a.omega;
  const Real cpi = (Real)a.cpi, spi = (Real)a.spi, scale = (Real)a.two_over_nt;
  // u lives in (vre, vim) between WaveHoltz iterations
  Real p[RY], pd[RY], vre[RY], vim[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) { vre[r] = 0; vim[r] = 0; }
  cluster.sync();  // every tile zeroed before any neighbour pushes into it

  __shared__ double red[2 * 32];
  __shared__ double part[2];
  __shared__ int stop_flag;
  int m_done = 0;
  // buffer parity runs on across WaveHoltz iterations: consecutive time steps
  // always alternate buffers (N_t - 1 may be odd), which the single barrier
  // per step relies on
  int cur = 0;
  for (int m = 0; m < a.m_wh; ++m) {
    const bool check = a.wh_tol > 0.0;
    if (check && active) {
#pragma unroll
      for (int r = 0; r < RY; ++r)
        if (j0 + r < nly) {
          stash[2 * ((j0 + r) * BW + il)] = vre[r];
          stash[2 * ((j0 + r) * BW + il) + 1] = vim[r];
        }
    }
    {
      const Vec4<Real> t0 = tab[0];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        p[r] = vre[r];
        pd[r] = omega * (vim[r] * cpi - vre[r] * spi);  // Re{-i w u e^{-i pi/N_t}}
        vre[r] = t0.z * p[r];
        vim[r] = t0.w * pd[r];
      }
    }
    for (int nu = 1; nu < a.Nt; ++nu) {
      const Vec4<Real> tb = tab[nu];
      Real* bufc = cur ? buf1 : buf0;
#pragma unroll
      for (int r = 0; r < RY; ++r) p[r] += sigma * pd[r];
      if (active) {
#pragma unroll
        for (int r = 0; r < RY; ++r) bufc[(j0 + r + P) * colsP + il + P] = p[r];
        if (push_left) {
          Real* dst = cur ? left1 : left0;
#pragma unroll
          for (int r = 0; r < RY; ++r) dst[(j0 + r + P) * colsP + BW + P + il] = p[r];
        }
        if (push_right) {
          Real* dst = cur ? right1 : right0;
#pragma unroll
          for (int r = 0; r < RY; ++r) dst[(j0 + r + P) * colsP + il - BW + P] = p[r];
        }
      }
      cluster.sync();
      // y: column values rows j0-P .. j0+RY
      Real col[RY + P + 1];
#pragma unroll
      for (int k = 0; k < P; ++k) col[k] = bufc[(j0 + k) * colsP + ile + P];
#pragma unroll
      for (int r = 0; r < RY; ++r) col[P + r] = p[r];
      col[P + RY] = bufc[(j0 + RY + P) * colsP + ile + P];
      Real sy[RY];
#pragma unroll
      for (int r = 0; r < RY; ++r) sy[r] = 0;
      {
        Real acc = 0;
#pragma unroll
        for (int b = 0; b <= P; ++b) acc += kref<Real>(a, P * (P + 1) + b) * col[b];
        sy[0] += bok * acc;
      }
#pragma unroll
      for (int qq = 0; qq < TY; ++qq) {
#pragma unroll
        for (int aa = 0; aa <= P; ++aa) {
          if (aa == P && qq == TY - 1) continue;  // belongs to the next strip
          Real acc = 0;
#pragma unroll
          for (int b = 0; b <= P; ++b) acc += kref<Real>(a, aa * (P + 1) + b) * col[P + qq * P + b];
          sy[qq * P + aa] += eok[qq] * acc;
        }
      }
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const Real* row = bufc + (j0 + r + P) * colsP + ile;
        Real sx = kx[P] * p[r];
#pragma unroll
        for (int tt = 0; tt < NK; ++tt) {
          if (tt == P) continue;
          sx += kx[tt] * row[tt];
        }
        const Real Ap = wy[r] * sx + wxy * sy[r];
        if (SRC) {
          pd[r] = alp[r] * pd[r] - bet[r] * Ap + bbr[r] * tb.x + bbi[r] * tb.y + gam[r] * p[r];
        } else {
          const int j = j0 + r;
          Real f = pd[r] - bet[r] * Ap;
          if (r % P == 0) {  // only element-boundary rows can be the first or last row
            if (j == 0) f += (al0 - Real(1)) * pd[r] + b0r * tb.x + b0i * tb.y + g0 * p[r];
            if (j == nly - 1) f += (alN - Real(1)) * pd[r] + bNr * tb.x + bNi * tb.y + gN * p[r];
          }
          if (edge_col && j > 0 && j < nly - 1) {
            const Vec4<Real> e = ecol[j * 2 + slot];
            f += e.x * pd[r] + e.y * tb.x + e.z * tb.y + e.w * p[r];
          }
          pd[r] = f;
        }
        vre[r] += tb.z * p[r];
        vim[r] += tb.w * pd[r];
      }
      cur ^= 1;
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      vre[r] *= scale;  // u^{(m+1)} = (2/N_t) v
      vim[r] *= scale;
    }
    m_done = m + 1;
    if (check) {
      double dn = 0.0, un = 0.0;
      if (active) {
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          if (j0 + r < nly) {
            const Real ox = stash[2 * ((j0 + r) * BW + il)], oy = stash[2 * ((j0 + r) * BW + il) + 1];
            const double dr = (double)vre[r] - ox, di = (double)vim[r] - oy;
            dn += dr * dr + di * di;
            un += (double)vre[r] * vre[r] + (double)vim[r] * vim[r];
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        un += __shfl_xor_sync(0xffffffffu, un, o);
      }
      const int warp = t >> 5, lane = t & 31;
      if (lane == 0) { red[2 * warp] = dn; red[2 * warp + 1] = un; }
      __syncthreads();
      if (t == 0) {
        double D = 0.0, U = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) { D += red[2 * w]; U += red[2 * w + 1]; }
        part[0] = D;
        part[1] = U;
      }
      cluster.sync();
      if (t == 0) {
        double D = 0.0, U = 0.0;
        for (int r = 0; r < CN; ++r) {  // same order on every CTA: identical decision
          const double* pr = cluster.map_shared_rank(part, r);
          D += pr[0];
          U += pr[1];
        }
        stop_flag = (D <= a.wh_tol * a.wh_tol * U) ? 1 : 0;
      }
      cluster.sync();  // remote reads of part[] done before it is rewritten
      if (stop_flag) break;
    }
  }

  // ---- epilogue: band-local u in shared memory, then outputs
  bool bad = false;
  Real* su = sm;  // [nly][BW] complex
  __syncthreads();
  if (active) {
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int j = j0 + r;
      if (j < nly) {
        su[2 * (j * BW + il)] = vre[r];
        su[2 * (j * BW + il) + 1] = vim[r];
        if (!isfinite(vre[r]) || !isfinite(vim[r])) bad = true;
        if (a.u_sub) {
          const int64_t n = (int64_t)l * nn + (int64_t)j * nlx + i;
          a.u_sub[2 * n] = (double)vre[r];
          a.u_sub[2 * n + 1] = (double)vim[r];
        }
      }
    }
  }
  if (bad) atomicOr(a.flags, 1);
  if (q == 0 && t == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  __syncthreads();
  const int NE = a.NE;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * NE;
  for (int k = t; k < 4 * NE; k += blockDim.x) {
    const int e = k / NE, tt = k % NE;
    // which CTA writes this slot entry: W edge + W/E padding -> band 0, E edge -> last band,
    // S/N edges -> the band holding column tt (padding past nlx -> last band)
    int owner;
    if (e == 0) owner = 0;
    else if (e == 1) owner = (tt < nly) ? CN - 1 : 0;
    else owner = (tt < nlx) ? tt / BW : CN - 1;
    if (owner != q) continue;
    const bool iface = (e == 0) ? ifW : (e == 1) ? ifE : (e == 2) ? ifS : ifN;
    const int len = (e < 2) ? nly : nlx;
    double* dst;
    if (iface) {
      const int r = (e == 0) ? l - 1 : (e == 1) ? l + 1 : (e == 2) ? l - a.Sx : l + a.Sx;
      dst = a.lam_out + 2 * (((int64_t)r * 4 + (e ^ 1)) * NE + tt);
    } else {
      dst = a.lam_out + 2 * (((int64_t)l * 4 + e) * NE + tt);
    }
    if (iface && tt < len) {
      const int gi = (e == 0) ? 0 : (e == 1) ? nlx - 1 : tt;
      const int gj = (e == 2) ? 0 : (e == 3) ? nly - 1 : tt;
      const int li = gi - i0;  // inside this band by the ownership rule
      const double ur = (double)su[2 * (gj * BW + li)], ui = (double)su[2 * (gj * BW + li) + 1];
      const double kk = kedgeL[e * NE + tt];
      const double lr = lamL[2 * (e * NE + tt)], li2 = lamL[2 * (e * NE + tt) + 1];
      // -lambda + 2 k (eta - i zeta) u  (eta = 0, zeta = 1: -lambda - 2ik u)
      dst[0] = -lr + 2.0 * kk * (a.eta * ur + a.zeta * ui);
      dst[1] = -li2 + 2.0 * kk * (a.eta * ui - a.zeta * ur);
    } else {
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  }
  cluster.sync();  // no CTA leaves while a neighbour may still touch its shared memory
}

template <typename Real, int P, int TY, int CN>
hz_status launch(SweepArgs a, int L, int BW, cudaStream_t st) {
  constexpr int RY = P * TY;
  const int threads = ((BW * a.NS + 31) / 32) * 32;
  if (threads > ClusterBlock<TY>::kMaxThreads) return HZ_ERR_UNSUPPORTED;
  const int rowsP = a.NS * RY + P + 1;
  const int colsP = BW + 2 * P;
  const size_t edge_off = (size_t)((2 * rowsP * colsP + 2 * a.nly * BW + 3) & ~3);  // Reals, as in the kernel
  size_t smem = edge_off * sizeof(Real) + (size_t)2 * a.nly * sizeof(Vec4<Real>);
  if (smem > 220 * 1024) return HZ_ERR_UNSUPPORTED;
  auto kern = a.rhs ? sweep_cluster_kernel<Real, P, TY, CN, true> : sweep_cluster_kernel<Real, P, TY, CN, false>;
  HZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(L * CN));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CN;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HZ_CUDA(cudaLaunchKernelEx(&cfg, kern, a, BW));
  note_launch();
  return HZ_OK;
}

template <typename Real, int P, int TY>
hz_status launch_TY(SweepArgs a, int L, cudaStream_t st) {
  // smallest cluster whose bands fit in one block
  a.NS = (a.nly + TY * P - 1) / (TY * P);
  for (int cn : {2, 4, 8}) {
    const int BW = (a.nlx + cn - 1) / cn;
    if (BW * (cn - 1) >= a.nlx || BW < P) continue;  // every band non-empty, halos within one band
    if (((BW * a.NS + 31) / 32) * 32 > ClusterBlock<TY>::kMaxThreads) continue;
    if (cn == 2) return launch<Real, P, TY, 2>(a, L, BW, st);
    if (cn == 4) return launch<Real, P, TY, 4>(a, L, BW, st);
    return launch<Real, P, TY, 8>(a, L, BW, st);
  }
  return HZ_ERR_UNSUPPORTED;
}

// Rows per thread 2P (a.ty_force != 4) or 4P (a.ty_force == 4, fewer and
// fuller threads: more work between cluster barriers).
template <typename Real, int P>
hz_status launch_P(SweepArgs a, int L, cudaStream_t st) {
  if (a.ty_force == 4) return launch_TY<Real, P, 4>(a, L, st);
  return launch_TY<Real, P, 2>(a, L, st);
}

template <typename Real>
hz_status launch_any(int P, const SweepArgs& a, int L, cudaStream_t st) {
  switch (P) {
    case 1: return launch_P<Real, 1>(a, L, st);
    case 2: return launch_P<Real, 2>(a, L, st);
    case 3: return launch_P<Real, 3>(a, L, st);
    case 4: return launch_P<Real, 4>(a, L, st);
    case 5: return launch_P<Real, 5>(a, L, st);
    case 6: return launch_P<Real, 6>(a, L, st);
    case 7: return launch_P<Real, 7>(a, L, st);
    default: return HZ_ERR_UNSUPPORTED;
  }
}

}  // namespace
}  // namespace cluster_sweep

}  // namespace hz
