// DD sweep on general convex quadrilaterals: Algorithm 1 (DDM cycle) on every
// subdomain, one thread block per subdomain, all subdomains in one launch
// (Sec. 6), with the element-form stiffness of Sec. 4 / Sec. 6.1 on mapped
// elements.
//
// Layout inside a block: thread t owns subdomain node t (column t % nlx, row
// t / nlx) and keeps its p, p-dot, filter sums and coefficients in registers;
// the (element, local node) pairs are spread over the threads in the same
// way (thread t takes pairs t, t + blockDim, ...).  Each time step:
//   1. p += sigma pd, published to shared memory; barrier;
//   2. per element node: the reference gradient (u_xi, u_eta) from P+1
//      neighbours each along the element's row and column, and the metric
//      fluxes F1 = w w (G11 u_xi + G12 u_eta), F2 = w w (G12 u_xi + G22 u_eta);
//      barrier;
//   3. per element node: its element's contribution to A p at that node,
//      sum_q D[q][a] F1(b, q) + sum_q D[q][b] F2(q, a); barrier;
//   4. per node: A p = the sum of the contributions of its (up to four)
//      elements (the assembly as a gather: no atomics), then the modified
//      leapfrog update and the filter sums.
// For P = 1 and 3 an element's (P+1)^2 nodes fill whole lanes of a warp:
// steps 2 and 3 are then one step, the contraction reading its element's
// fluxes by warp shuffles, and a time step has two barriers.
// Splitting the contraction (3) from the gather (4) keeps the work per thread
// the same for every node (a cross point gathers four values, not four
// contractions); element arrays in shared memory use an odd stride per
// element so that neighbouring elements fall in different banks.  The metric
// (3 values per element node) stays in registers when every thread owns at
// most one element node, else it is read from shared memory.
// Prologue and epilogue (right-hand side from the split global source and
// the incoming lambda with arc-length edge weights, WaveHoltz stopping test,
// transmission update into the neighbours' slots) follow the Cartesian block
// kernel.
#include <cuda_runtime.h>

#include <cmath>

#include "hz_internal.h"

namespace hz {
namespace {

template <typename Real>
struct MTab4;
template <>
struct MTab4<float> {
  using type = float4;
};
struct alignas(32) MDbl4 {
  double x, y, z, w;
};
template <>
struct MTab4<double> {
  using type = MDbl4;
};

constexpr int kMappedThreads = 1024;

// element stride in shared memory: (P+1)^2 rounded up to an odd count
template <int P>
struct MappedStride {
  static constexpr int value = ((P + 1) * (P + 1)) | 1;
};

template <typename Real, int P>
__global__ void __launch_bounds__(kMappedThreads) sweep_mapped_kernel(const __grid_constant__ MappedSweepArgs ma) {
  constexpr int M = P + 1, N2 = M * M, S = MappedStride<P>::value;
  constexpr bool kWarpElem = (32 % N2) == 0;  // whole elements per warp (P = 1, 3)
  using Tab = typename MTab4<Real>::type;
  const SweepArgs& a = ma.base;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nlx = a.nlx, nly = a.nly, nl = nlx * nly;
  const int snx = ma.snx, sny = ma.sny;
  const int nel = snx * sny, Ne = nel * N2;
  Real* ps = reinterpret_cast<Real*>(smem_raw);  // [nl]
  Real* f1 = ps + nl;                            // [nel][S]
  Real* f2 = f1 + nel * S;                       // [nel][S]
  Real* cc = f2 + nel * S;                       // [nel][S] element contributions to A p
  Real* geo = cc + nel * S;                      // [Ne][3]
  __shared__ Real Ds[N2];
  __shared__ double red[2 * 32];
  __shared__ int stop_flag;

  const int l = sweep_subdomain(ma.base, blockIdx.x), t = threadIdx.x;
  const int sxi = l % a.Sx, syi = l / a.Sx;
  for (int k = t; k < N2; k += blockDim.x) Ds[k] = Real(ma.D[k]);
  {
    const Real* g = static_cast<const Real*>(ma.geo) + (int64_t)l * Ne * 3;
    for (int k = t; k < 3 * Ne; k += blockDim.x) geo[k] = g[k];
  }
  const bool own = t < nl;
  const int i = own ? t % nlx : 0, j = own ? t / nlx : 0;
  // element slots of the node's (up to four) elements: in x the one on the
  // left (local index P) and the one it starts (local index i % P), likewise
  // in y; unused slots are -1
  int slot[4] = {-1, -1, -1, -1};
  if (own) {
    int ex[2], ax[2], nex = 0, ey[2], by[2], ney = 0;
    if (i % P == 0 && i > 0) { ex[nex] = i / P - 1; ax[nex] = P; ++nex; }
    if (i / P < snx) { ex[nex] = i / P; ax[nex] = i % P; ++nex; }
    if (j % P == 0 && j > 0) { ey[ney] = j / P - 1; by[ney] = P; ++ney; }
    if (j / P < sny) { ey[ney] = j / P; by[ney] = j % P; ++ney; }
    int q = 0;
    for (int qy = 0; qy < ney; ++qy)
      for (int qx = 0; qx < nex; ++qx) slot[q++] = (ey[qy] * snx + ex[qx]) * S + by[qy] * M + ax[qx];
  }
  // the thread's element node when it owns at most one (metric in registers)
  const bool one_en = Ne <= (int)blockDim.x;
  const bool own_en = t < Ne;
  Real g0 = Real(0), g1 = Real(0), g2 = Real(0);
  int en_e = 0, en_b = 0, en_a = 0;
  if (own_en) {
    en_e = t / N2;
    const int loc = t - en_e * N2;
    en_b = loc / M;
    en_a = loc - en_b * M;
  }
  __syncthreads();
  // one element node per thread: its metric, its rows of D (gradient) and its
  // columns of D (contraction) in registers, its shared-memory addresses fixed
  Real Dar[M], Dbr[M], Dac[M], Dbc[M];
  int rowo = 0, colo = 0, f1o = 0, f2o = 0, kown = 0;  // offsets into ps, f1, f2
  if (one_en && own_en) {
    g0 = geo[3 * t];
    g1 = geo[3 * t + 1];
    g2 = geo[3 * t + 2];
    const int exe = en_e % snx, eye = en_e / snx;
    rowo = (eye * P + en_b) * nlx + exe * P;
    colo = (eye * P) * nlx + exe * P + en_a;
    f1o = en_e * S + en_b * M;
    f2o = en_e * S + en_a;
    kown = en_e * S + en_b * M + en_a;
  }
  const int lbase = (t & 31) - (en_b * M + en_a);  // lane of the thread's element node (0, 0)
#pragma unroll
  for (int c = 0; c < M; ++c) {
    Dar[c] = Ds[en_a * M + c];
    Dbr[c] = Ds[en_b * M + c];
    Dac[c] = Ds[c * M + en_a];
    Dbc[c] = Ds[c * M + en_b];
  }

  // ---- per-node coefficients and right-hand side (Algorithm 1 step 1)
  const int64_t nn = (int64_t)nl;
  const bool ifW = sxi > 0, ifE = sxi < a.Sx - 1, ifS = syi > 0, ifN = syi < a.Sy - 1;
  const double* lamL = a.lam_in + (int64_t)l * 4 * a.NE * 2;
  const double* kedgeL = a.kedge + (int64_t)l * 4 * a.NE;
  const double* wE = ma.wedge + (int64_t)l * 4 * a.NE;
  Real bet = Real(0), alp = Real(0), bbr = Real(0), bbi = Real(0), gam = Real(0);
  if (own) {
    const int64_t n = (int64_t)j * nlx + i;
    const double be = (double)static_cast<const Real*>(a.beta)[(int64_t)l * nn + n];
    const double al = (double)static_cast<const Real*>(a.alpha)[(int64_t)l * nn + n];
    double br = 0.0, bi = 0.0, hm = 0.0;
    if (a.rhs) {
      const double sh = ma.share[(int64_t)l * nn + n];
      const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
      br = sh * a.rhs[2 * (J * a.NXg + I)];
      bi = sh * a.rhs[2 * (J * a.NXg + I) + 1];
    }
    auto edge = [&](int e, int q) {
      const double wq = wE[e * a.NE + q];
      br += wq * lamL[2 * (e * a.NE + q)];
      bi += wq * lamL[2 * (e * a.NE + q) + 1];
      hm += wq * kedgeL[e * a.NE + q];
    };
    if (i == 0 && ifW) edge(0, j);
    if (i == nlx - 1 && ifE) edge(1, j);
    if (j == 0 && ifS) edge(2, i);
    if (j == nly - 1 && ifN) edge(3, i);
    gam = Real(-be * a.eta * hm);  // interface boundary mass, -beta w eta <c^-1 phi, phi>
    bet = Real(be);
    alp = Real(al);
    bbr = Real(be * br);
    bbi = Real(be * bi);
  }
  const Tab* tab = static_cast<const Tab*>(a.tab);
  const Real sigma = Real(a.sigma), omega = Real(a.omega);
  const Real cpi = Real(a.cpi), spi = Real(a.spi), scale = Real(a.two_over_nt);
  Real ure = Real(0), uim = Real(0);
  if (a.u0 && own) {  // warm start from a previous sweep's subdomain solution
    const int64_t n = (int64_t)l * nn + t;
    ure = Real(a.u0[2 * n]);
    uim = Real(a.u0[2 * n + 1]);
  }
  __syncthreads();

  int m_done = 0;
  for (int m = 0; m < a.m_wh; ++m) {
    const Tab t0 = tab[0];
    Real p = ure;
    Real pd = omega * (uim * cpi - ure * spi);  // Re{-i w u e^{-i pi/N_t}}
    Real vre = t0.z * p, vim = t0.w * pd;
    for (int nu = 1; nu < a.Nt; ++nu) {
      const Tab tb = tab[nu];
      p += sigma * pd;
      if (own) ps[t] = p;
      __syncthreads();
      if (kWarpElem && one_en) {
        // 2+3 fused: an element's (P+1)^2 nodes are lanes of one warp, so the
        // contraction reads the fluxes of its element by shuffles (no
        // shared-memory round trip, one barrier less per step)
        Real f1v = Real(0), f2v = Real(0);
        if (own_en) {
          Real uxi = Real(0), ueta = Real(0);
#pragma unroll
          for (int c = 0; c < M; ++c) {
            uxi += Dar[c] * ps[rowo + c];
            ueta += Dbr[c] * ps[colo + c * nlx];
          }
          f1v = g0 * uxi + g1 * ueta;
          f2v = g1 * uxi + g2 * ueta;
        }
        Real acc = Real(0);
#pragma unroll
        for (int q = 0; q < M; ++q)
          acc += Dac[q] * __shfl_sync(0xffffffffu, f1v, lbase + en_b * M + q) +
                 Dbc[q] * __shfl_sync(0xffffffffu, f2v, lbase + q * M + en_a);
        if (own_en) cc[kown] = acc;
      } else {
        // 2. metric fluxes per element node
        if (one_en) {
          if (own_en) {
            Real uxi = Real(0), ueta = Real(0);
#pragma unroll
            for (int c = 0; c < M; ++c) {
              uxi += Dar[c] * ps[rowo + c];
              ueta += Dbr[c] * ps[colo + c * nlx];
            }
            f1[kown] = g0 * uxi + g1 * ueta;
            f2[kown] = g1 * uxi + g2 * ueta;
          }
        } else {
          for (int en = t; en < Ne; en += blockDim.x) {
            const int e = en / N2, loc = en - e * N2;
            const int b = loc / M, aa = loc - b * M;
            const int exe = e % snx, eye = e / snx;
            const Real* row = ps + (eye * P + b) * nlx + exe * P;
            const Real* col = ps + (eye * P) * nlx + exe * P + aa;
            Real uxi = Real(0), ueta = Real(0);
#pragma unroll
            for (int c = 0; c < M; ++c) {
              uxi += Ds[aa * M + c] * row[c];
              ueta += Ds[b * M + c] * col[c * nlx];
            }
            const Real* g = geo + 3 * en;
            f1[e * S + loc] = g[0] * uxi + g[1] * ueta;
            f2[e * S + loc] = g[1] * uxi + g[2] * ueta;
          }
        }
        __syncthreads();
        // 3. element contributions D^T F per element node
        if (one_en) {
          if (own_en) {
            Real acc = Real(0);
#pragma unroll
            for (int q = 0; q < M; ++q) acc += Dac[q] * f1[f1o + q] + Dbc[q] * f2[f2o + q * M];
            cc[kown] = acc;
          }
        } else
        for (int en = t; en < Ne; en += blockDim.x) {
          const int e = en / N2, loc = en - e * N2;
          const int b = loc / M, aa = loc - b * M;
          const Real* F1 = f1 + e * S + b * M;  // F1(b, q)
          const Real* F2 = f2 + e * S + aa;     // F2(q, aa), stride M
          Real acc = Real(0);
#pragma unroll
          for (int q = 0; q < M; ++q) acc += Ds[q * M + aa] * F1[q] + Ds[q * M + b] * F2[q * M];
          cc[e * S + loc] = acc;
        }
      }
      __syncthreads();
      // 4. gather per node, leapfrog update
      if (own) {
        Real Ap = cc[slot[0]];
#pragma unroll
        for (int q = 1; q < 4; ++q)
          if (slot[q] >= 0) Ap += cc[slot[q]];
        pd = alp * pd - bet * Ap + bbr * tb.x + bbi * tb.y + gam * p;
        vre += tb.z * p;
        vim += tb.w * pd;
      }
    }
    // u^{(m+1)} = (2/N_t) v; FP64 norms of the update only in tolerance mode
    const Real nr = scale * vre, ni = scale * vim;
    double dn = 0.0, un = 0.0;
    const bool check = a.wh_tol > 0.0;
    if (check && own) {
      const double dr = (double)nr - (double)ure, di = (double)ni - (double)uim;
      dn = dr * dr + di * di;
      un = (double)nr * nr + (double)ni * ni;
    }
    if (own) {
      ure = nr;
      uim = ni;
    }
    m_done = m + 1;
    if (check) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        un += __shfl_xor_sync(0xffffffffu, un, o);
      }
      const int warp = t >> 5, lane = t & 31;
      if (lane == 0) {
        red[2 * warp] = dn;
        red[2 * warp + 1] = un;
      }
      __syncthreads();
      if (t == 0) {
        double Dn = 0.0, Un = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
          Dn += red[2 * w];
          Un += red[2 * w + 1];
        }
        stop_flag = (Dn <= a.wh_tol * a.wh_tol * Un) ? 1 : 0;
      }
      __syncthreads();
      if (stop_flag) break;
    }
    __syncthreads();
  }

  // ---- epilogue: outputs (u of the subdomain staged in shared memory)
  Real* su = ps;  // [nl] x 2 fits in ps + f1 (Ne >= nl)
  __syncthreads();
  bool bad = false;
  if (own) {
    const int64_t n = t;
    su[2 * n] = ure;
    su[2 * n + 1] = uim;
    if (!isfinite((double)ure) || !isfinite((double)uim)) bad = true;
    if (a.u_sub) {
      a.u_sub[2 * ((int64_t)l * nn + n)] = (double)ure;
      a.u_sub[2 * ((int64_t)l * nn + n) + 1] = (double)uim;
    }
  }
  if (bad) atomicOr(a.flags, 1);
  if (t == 0 && a.wh_iter_max) {
    atomicMax(a.wh_iter_max, m_done);
    atomicAdd(a.wh_iter_sum, (unsigned long long)m_done);
  }
  __syncthreads();
  const int NE = a.NE;
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
        // -lambda + 2 k (eta - i zeta) u
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

template <typename Real, int P>
hz_status launch_mapped_P(const MappedSweepArgs& a, int L, cudaStream_t st) {
  constexpr int N2 = (P + 1) * (P + 1), S = MappedStride<P>::value;
  const int nl = a.base.nlx * a.base.nly;
  const int nel = a.snx * a.sny, Ne = nel * N2;
  if (nl > kMappedThreads) return fail(HZ_ERR_UNSUPPORTED, "mapped sweep: subdomain has more than 1024 nodes");
  int threads = nl > Ne ? nl : Ne;
  if (threads > kMappedThreads) threads = kMappedThreads;
  threads = (threads + 31) / 32 * 32;
  const size_t smem = ((size_t)nl + 3 * (size_t)nel * S + 3 * (size_t)Ne) * sizeof(Real);
  if (smem > 200 * 1024) return fail(HZ_ERR_UNSUPPORTED, "mapped sweep: subdomain exceeds shared memory");
  auto kern = sweep_mapped_kernel<Real, P>;
  if (smem > 48 * 1024) HZ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<L, threads, smem, st>>>(a);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

template <typename Real>
hz_status launch_mapped_T(int P, const MappedSweepArgs& a, int L, cudaStream_t st) {
  switch (P) {
    case 1: return launch_mapped_P<Real, 1>(a, L, st);
    case 2: return launch_mapped_P<Real, 2>(a, L, st);
    case 3: return launch_mapped_P<Real, 3>(a, L, st);
    case 4: return launch_mapped_P<Real, 4>(a, L, st);
    case 5: return launch_mapped_P<Real, 5>(a, L, st);
    case 6: return launch_mapped_P<Real, 6>(a, L, st);
    case 7: return launch_mapped_P<Real, 7>(a, L, st);
    default: return fail(HZ_ERR_UNSUPPORTED, "degree outside 1..7");
  }
}

}  // namespace
}  // namespace hz
