// DD sweep kernel: Algorithm 1 (DDM cycle) on every subdomain, one thread
// block per subdomain, all subdomains in one launch (Sec. 6).
//
// Layout inside a block (subdomain of nlx x nly GLL nodes, structured):
//   thread t owns column i = t % nlx and a strip of RY = P*TY rows starting
//   at row j0 = (t / nlx) * RY (strips are aligned to element rows, so the
//   row position inside an element is a compile-time constant).  Rows past
//   nly are dead (zero state, zero coefficients).
//   The strip's p, p-dot, v (= u in place), beta, alpha and beta*b live in
//   registers for the whole WaveHoltz loop; p is published each time step to
//   a double-buffered shared-memory tile with a zero halo of P nodes, which
//   makes one block barrier per time step sufficient.
//
// Stiffness apply (Sec. 4, A_ij = (grad phi_j, grad phi_i), GLL quadrature):
//   on a Cartesian element grid the collocated-GLL stiffness is
//   A = Kx (x) Wy + Wx (x) Ky with Kx, Ky the assembled 1D stiffness and
//   Wx, Wy the lumped 1D weights, so (A p)_ij = Wy_j (Kx p)_ij + Wx_i (Ky p)_ij.
//   x: per-lane assembled row of Kx (2P+1 taps, one-sided at subdomain ends)
//      against neighbours in shared memory;
//   y: element by element over the strip's elements from registers (the
//      element's 1D reference stiffness Kref is a kernel parameter, so its
//      entries are constant-bank operands), plus the element below the strip.
//   This replaces the paper's element-local gradient/atomic form (Sec. 6.1)
//   by the assembled tensor-product form: no duplicated element nodes, no
//   atomics, one barrier per step.
//
// Time loop (Sec. 5, modified leapfrog and eq. (WaveHoltz) with the
// -1/(i omega) filter sign and 2/N_t scaling):
//   p += sigma pd;  pd = alpha pd + beta(-A p + Re{b e^{-2 pi i nu/N_t}});
//   v_re += kappa_nu p;  v_im += (kappa_{nu+1/2}/omega) pd.
// Epilogue: lambda_{r,l} = -lambda_{l,r} - 2 i (omega/c) u_l on each
// interface (eq. (lambda-iteration), sign read as -2ik), written into the
// neighbour's slot; slots of outer edges are zeroed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "hz_internal.h"

// Included by hz_sweep_f32.cu / hz_sweep_f64.cu with HZ_SWEEP_REAL and
// HZ_SWEEP_LAUNCHER defined (one precision per translation unit).

namespace hz {
namespace {

template <typename Real>
struct Tab4T;
template <>
struct Tab4T<float> {
  using type = float4;
};
struct alignas(32) Dbl4 {
  double x, y, z, w;
};
template <>
struct Tab4T<double> {
  using type = Dbl4;
};

// 16-bit storage trials: the wave state is rounded to FP16 / BF16 after every
// update (the filter sums stay in the working precision).
template <typename Real>
__device__ __forceinline__ Real round16(Real v, int mode) {
  if (mode == 1) return Real(__half2float(__float2half_rn((float)v)));
  if (mode == 2) return Real(__bfloat162float(__float2bfloat16_rn((float)v)));
  return v;
}

template <typename Real>
__device__ __forceinline__ Real kref(const SweepArgs& a, int k);
template <>
__device__ __forceinline__ float kref<float>(const SweepArgs& a, int k) { return a.Kref32[k]; }
template <>
__device__ __forceinline__ double kref<double>(const SweepArgs& a, int k) { return a.Kref[k]; }

template <typename Real, int P, int TY, int MAXT>
__global__ void __launch_bounds__(MAXT) sweep_kernel(const __grid_constant__ SweepArgs a) {
  constexpr int RY = P * TY;
  constexpr int NK = 2 * P + 1;
  using Tab = typename Tab4T<Real>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* sm = reinterpret_cast<Real*>(smem_raw);

  const int l = sweep_subdomain(a, blockIdx.x);
  const int sxi = l % a.Sx, syi = l / a.Sx;
  const int nlx = a.nlx, nly = a.nly;
  const int t = threadIdx.x;
  const int i = t % nlx;
  const int s = t / nlx;
  const bool active = s < a.NS;
  const int se = active ? s : 0;  // inactive threads read a valid strip, never write
  const int j0 = se * RY;
  const int colsP = nlx + 2 * P;
  const int rowsP = a.NS * RY + P + 1;
  const int PS = rowsP * colsP;
  Real* buf0 = sm;
  Real* buf1 = sm + PS;

  for (int k = t; k < 2 * PS; k += blockDim.x) sm[k] = Real(0);

  // ---- per-lane x stencil (assembled 1D row, scaled by 2/hx) and weights
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
    kx[tt] = Real(v * a.kxs);
  }
  const Real wxy = Real(a.kys * a.hx2 * ((own_x ? a.w[ax] : 0.0) + (left_x ? a.w[P] : 0.0)));
  Real wy[RY];
  Real eok[TY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int ay = r % P;
    const int ey = (j0 + r) / P;
    const bool own_y = ey < a.sye;
    const bool below_y = (ay == 0) && (ey >= 1);
    wy[r] = Real(a.hy2 * ((own_y ? a.w[ay] : 0.0) + (below_y ? a.w[P] : 0.0)));
  }
#pragma unroll
  for (int q = 0; q < TY; ++q) eok[q] = (se * TY + q < a.sye) ? Real(1) : Real(0);
  const Real bok = (se > 0) ? Real(1) : Real(0);

  // ---- per-node coefficients and right-hand side (assembled from the split
  // global source and the incoming transmission data, Algorithm 1 step 1)
  const int64_t nn = (int64_t)nlx * nly;
  const Real* betaG = static_cast<const Real*>(a.beta) + (int64_t)l * nn;
  const Real* alphaG = static_cast<const Real*>(a.alpha) + (int64_t)l * nn;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  const double* kedgeE = a.kedge + (int64_t)l * 4 * a.NE;
  Real bet[RY], alp[RY], bbr[RY], bbi[RY], gam[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = j0 + r;
    const bool live = active && (j < nly);
    double be = 0.0, al = 0.0, br = 0.0, bi = 0.0, hm = 0.0;
    if (live) {
      const int64_t n = (int64_t)j * nlx + i;
      be = (double)betaG[n];
      al = (double)alphaG[n];
      if (a.rhs) {
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
    gam[r] = Real(-be * a.eta * hm);  // gamma = -beta w eta <c^-1 phi, phi>
    bet[r] = Real(be);
    alp[r] = Real(al);
    bbr[r] = Real(be * br);
    bbi[r] = Real(be * bi);
  }

  const Tab* tab = static_cast<const Tab*>(a.tab);
  const Real sigma = Real(a.sigma), omega = Real(a.omega);
  const Real cpi = Real(a.cpi), spi = Real(a.spi), scale = Real(a.two_over_nt);
  Real ure[RY], uim[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    ure[r] = Real(0);
    uim[r] = Real(0);
    const int j = j0 + r;
    if (a.u0 && active && j < nly) {  // warm start from a previous sweep's subdomain solution
      const int64_t n = (int64_t)l * nn + (int64_t)j * nlx + i;
      ure[r] = Real(a.u0[2 * n]);
      uim[r] = Real(a.u0[2 * n + 1]);
    }
  }
  __syncthreads();

  __shared__ double red[2 * 32];
  __shared__ int stop_flag;
  int m_done = 0;
  // buffer parity runs on across WaveHoltz iterations: consecutive time steps
  // always alternate buffers (N_t - 1 may be odd), which the single barrier
  // per step relies on
  int cur = 0;
  for (int m = 0; m < a.m_wh; ++m) {
    Real p[RY], pd[RY], vre[RY], vim[RY];
    {
      const Tab t0 = tab[0];
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        p[r] = ure[r];
        pd[r] = omega * (uim[r] * cpi - ure[r] * spi);  // Re{-i w u e^{-i pi/N_t}}
        vre[r] = t0.z * p[r];
        vim[r] = t0.w * pd[r];
      }
    }
    for (int nu = 1; nu < a.Nt; ++nu) {
      const Tab tb = tab[nu];
      Real* bufc = cur ? buf1 : buf0;
#pragma unroll
      for (int r = 0; r < RY; ++r) p[r] += sigma * pd[r];
      if (a.round_mode) {
#pragma unroll
        for (int r = 0; r < RY; ++r) p[r] = round16(p[r], a.round_mode);
      }
      if (active) {
#pragma unroll
        for (int r = 0; r < RY; ++r) bufc[(j0 + r + P) * colsP + i + P] = p[r];
      }
      __syncthreads();
      // y: column values rows j0-P .. j0+RY
      Real col[RY + P + 1];
#pragma unroll
      for (int k = 0; k < P; ++k) col[k] = bufc[(j0 + k) * colsP + i + P];
#pragma unroll
      for (int r = 0; r < RY; ++r) col[P + r] = p[r];
      col[P + RY] = bufc[(j0 + RY + P) * colsP + i + P];
      Real sy[RY];
#pragma unroll
      for (int r = 0; r < RY; ++r) sy[r] = Real(0);
      {  // element below the strip -> its top node (strip row 0)
        Real acc = Real(0);
#pragma unroll
        for (int b = 0; b <= P; ++b) acc += kref<Real>(a, P * (P + 1) + b) * col[b];
        sy[0] += bok * acc;
      }
#pragma unroll
      for (int q = 0; q < TY; ++q) {
#pragma unroll
        for (int aa = 0; aa <= P; ++aa) {
          if (aa == P && q == TY - 1) continue;  // belongs to the next strip
          Real acc = Real(0);
#pragma unroll
          for (int b = 0; b <= P; ++b) acc += kref<Real>(a, aa * (P + 1) + b) * col[P + q * P + b];
          sy[q * P + aa] += eok[q] * acc;
        }
      }
      // x: assembled row against shared-memory neighbours
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const Real* row = bufc + (j0 + r + P) * colsP + i;
        Real sx = kx[P] * p[r];
#pragma unroll
        for (int tt = 0; tt < NK; ++tt) {
          if (tt == P) continue;
          sx += kx[tt] * row[tt];
        }
        const Real Ap = wy[r] * sx + wxy * sy[r];
        pd[r] = round16(alp[r] * pd[r] - bet[r] * Ap + bbr[r] * tb.x + bbi[r] * tb.y + gam[r] * p[r], a.round_mode);
        vre[r] += tb.z * p[r];
        vim[r] += tb.w * pd[r];
      }
      cur ^= 1;
    }
    // u^{(m+1)} = (2/N_t) v; FP64 norms of the update only in tolerance mode
    double dn = 0.0, un = 0.0;
    const bool check = a.wh_tol > 0.0;
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const Real nr = scale * vre[r], ni = scale * vim[r];
      if (check) {
        const double dr = (double)nr - (double)ure[r], di = (double)ni - (double)uim[r];
        dn += dr * dr + di * di;
        un += (double)nr * nr + (double)ni * ni;
      }
      ure[r] = nr;
      uim[r] = ni;
    }
    m_done = m + 1;
    if (check) {
      // block reduction of ||u^{m+1}-u^m||^2 and ||u^{m+1}||^2 (dead nodes are 0)
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
        for (int wI = 0; wI < (int)(blockDim.x + 31) / 32; ++wI) { D += red[2 * wI]; U += red[2 * wI + 1]; }
        stop_flag = (D <= a.wh_tol * a.wh_tol * U) ? 1 : 0;
      }
      __syncthreads();
      if (stop_flag) break;
    }
    __syncthreads();
  }

  // ---- epilogue: outputs
  bool bad = false;
  Real* su = sm;  // complex u of the subdomain, [nly][nlx] x 2
  __syncthreads();
  if (active) {
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const int j = j0 + r;
      if (j < nly) {
        const int64_t n = (int64_t)j * nlx + i;
        su[2 * n] = ure[r];
        su[2 * n + 1] = uim[r];
        if (!isfinite((double)ure[r]) || !isfinite((double)uim[r])) bad = true;
        if (a.u_sub) {
          a.u_sub[2 * ((int64_t)l * nn + n)] = (double)ure[r];
          a.u_sub[2 * ((int64_t)l * nn + n) + 1] = (double)uim[r];
        }
      }
    }
  }
  if (bad) atomicOr(a.flags, 1);
  if (t == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  __syncthreads();
  const int NE = a.NE;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * NE;
  for (int k = t; k < 4 * NE; k += blockDim.x) {
    const int e = k / NE, tt = k % NE;
    const bool iface = (e == 0) ? ifW : (e == 1) ? ifE : (e == 2) ? ifS : ifN;
    const int len = (e < 2) ? nly : nlx;
    if (iface) {
      const int r = (e == 0) ? l - 1 : (e == 1) ? l + 1 : (e == 2) ? l - a.Sx : l + a.Sx;
      const int opp = e ^ 1;
      double* dst = a.lam_out + 2 * (((int64_t)r * 4 + opp) * NE + tt);
      if (tt < len) {
        const int ii = (e == 0) ? 0 : (e == 1) ? nlx - 1 : tt;
        const int jj = (e == 2) ? 0 : (e == 3) ? nly - 1 : tt;
        const int64_t n = (int64_t)jj * nlx + ii;
        const double ur = (double)su[2 * n], ui = (double)su[2 * n + 1];
        const double kk = kedgeL[e * NE + tt];
        const double lr = lamL[2 * (e * NE + tt)], li = lamL[2 * (e * NE + tt) + 1];
        // -lambda + 2 k (eta - i zeta) u  (eta = 0, zeta = 1: -lambda - 2ik u)
        dst[0] = -lr + 2.0 * kk * (a.eta * ur + a.zeta * ui);
        dst[1] = -li + 2.0 * kk * (a.eta * ui - a.zeta * ur);
      } else {
        dst[0] = 0.0;
        dst[1] = 0.0;
      }
    } else {
      double* dst = a.lam_out + 2 * (((int64_t)l * 4 + e) * NE + tt);
      dst[0] = 0.0;
      dst[1] = 0.0;
    }
  }
}

template <typename Real, int P, int TY>
hz_status launch_one(const SweepArgs& a, int L, cudaStream_t st) {
  constexpr int RY = P * TY;
  const int threads = ((a.nlx * a.NS + 31) / 32) * 32;
  if (threads > 1024) return fail(HZ_ERR_UNSUPPORTED, "subdomain too large for one thread block");
  const int rowsP = a.NS * RY + P + 1;
  const int colsP = a.nlx + 2 * P;
  size_t smem = (size_t)2 * rowsP * colsP * sizeof(Real);
  const size_t need_u = (size_t)2 * a.nlx * a.nly * sizeof(Real);
  if (need_u > smem) smem = need_u;
  if (smem > 200 * 1024) return fail(HZ_ERR_UNSUPPORTED, "subdomain tile exceeds shared memory");
  if (threads <= 256) {
    auto kern = sweep_kernel<Real, P, TY, 256>;
    if (smem > 48 * 1024) HZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<L, threads, smem, st>>>(a);
    note_launch();
  } else {
    auto kern = sweep_kernel<Real, P, TY, 1024>;
    if (smem > 48 * 1024) HZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<L, threads, smem, st>>>(a);
    note_launch();
  }
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

template <typename Real, int P>
hz_status launch_P(SweepArgs a, int L, cudaStream_t st) {
  // rows per thread: P (TY = 1) when it fits in 1024 threads, else 2P;
  // a.ty_force (autotuner) selects one explicitly
  if (a.ty_force != 2) {
    a.NS = (a.nly + P - 1) / P;
    if (a.nlx * a.NS <= 1024) return launch_one<Real, P, 1>(a, L, st);
    if (a.ty_force == 1) return HZ_ERR_UNSUPPORTED;
  }
  a.NS = (a.nly + 2 * P - 1) / (2 * P);
  if (a.nlx * a.NS <= 1024) return launch_one<Real, P, 2>(a, L, st);
  return fail(HZ_ERR_UNSUPPORTED, "subdomain too large for the one-block sweep");
}

}  // namespace

hz_status HZ_SWEEP_LAUNCHER(int P, const SweepArgs& a, int L, cudaStream_t st) {
  switch (P) {
    case 1: return launch_P<HZ_SWEEP_REAL, 1>(a, L, st);
    case 2: return launch_P<HZ_SWEEP_REAL, 2>(a, L, st);
    case 3: return launch_P<HZ_SWEEP_REAL, 3>(a, L, st);
    case 4: return launch_P<HZ_SWEEP_REAL, 4>(a, L, st);
    case 5: return launch_P<HZ_SWEEP_REAL, 5>(a, L, st);
    case 6: return launch_P<HZ_SWEEP_REAL, 6>(a, L, st);
    case 7: return launch_P<HZ_SWEEP_REAL, 7>(a, L, st);
    default: return fail(HZ_ERR_UNSUPPORTED, "degree outside 1..7");
  }
}

}  // namespace hz
