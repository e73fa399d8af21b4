// FP64 kernels around the sweep: leapfrog coefficients, right-hand side,
// global operator residual, assembly of subdomain copies, and the vector
// operations of the outer Krylov iteration.  All stream their data once with
// coalesced x-fastest access.  The right-hand side and the assembly are
// HBM-bound; the residual and the Krylov vector kernels do enough FP64
// arithmetic per byte that this part's FP64 pipe bounds them, so they are
// written with the fewest FP64 operations (FMA chains).  Reductions are
// two-pass with a fixed summation order (deterministic results).
#include <cuda_runtime.h>

#include <atomic>

#include <cmath>

#include "hz_internal.h"

namespace hz {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of NV values per thread into out[0..NV-1] (thread 0 holds result).
template <int NV>
__device__ void block_sum(double (&v)[NV], double* out) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = (lane < nw) ? sh[k][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0) out[k] = x;
    }
  }
}

// ---- leapfrog coefficients (Sec. 5): per subdomain node
//   M = W / c^2 (W = Wx_i Wy_j, or the mapped mesh's lumped weight),
//   H = (edge weights over all four subdomain edges) / c
//   alpha = (M - theta H)/(M + theta H), beta = sigma/(M + theta H)
__global__ void prepare_kernel(const __grid_constant__ PrepArgs a) {
  const int l = blockIdx.y;
  const int nn = a.nlx * a.nly;
  const int sxi = l % a.Sx, syi = l / a.Sx;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += gridDim.x * blockDim.x) {
    const int i = n % a.nlx, j = n / a.nlx;
    const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
    const double c = a.c[J * a.NXg + I];
    // lumped weight and edge weights: products of the 1D tables on a Cartesian
    // mesh, the map's per-node values on a mapped one
    const double* E = a.Esub ? a.Esub + (int64_t)l * 4 * a.NE : nullptr;
    const double W = a.Wsub ? a.Wsub[(int64_t)l * nn + n] : a.wxs[i] * a.wys[j];
    const double eS = E ? E[2 * a.NE + i] : a.wxs[i], eN = E ? E[3 * a.NE + i] : a.wxs[i];
    const double eW = E ? E[0 * a.NE + j] : a.wys[j], eE = E ? E[1 * a.NE + j] : a.wys[j];
    const double M = W / (c * c);
    // impedance damping on every subdomain edge: weight 1 on the outer
    // boundary, zeta on interfaces (the interface condition's d_t part)
    const double fS = syi > 0 ? a.zeta : 1.0, fN = syi < a.Sy - 1 ? a.zeta : 1.0;
    const double fW = sxi > 0 ? a.zeta : 1.0, fE = sxi < a.Sx - 1 ? a.zeta : 1.0;
    const double Hw = (j == 0 ? fS * eS : 0.0) + (j == a.nly - 1 ? fN * eN : 0.0) + (i == 0 ? fW * eW : 0.0) +
                      (i == a.nlx - 1 ? fE * eE : 0.0);
    const double H = Hw / c;
    const double den = M + a.theta * H;
    const double be = a.sigma / den;
    const double al = (M - a.theta * H) / den;
    const int64_t k = (int64_t)l * nn + n;
    a.beta64[k] = be;
    a.alpha64[k] = al;
    a.beta32[k] = (float)be;
    a.alpha32[k] = (float)al;
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < 4 * a.NE; k += blockDim.x) {
      const int e = k / a.NE, t = k % a.NE;
      const int len = (e < 2) ? a.nly : a.nlx;
      double val = 0.0;
      if (t < len) {
        const int i = (e == 0) ? 0 : (e == 1) ? a.nlx - 1 : t;
        const int j = (e == 2) ? 0 : (e == 3) ? a.nly - 1 : t;
        const int64_t I = (int64_t)sxi * a.snxP + i, J = (int64_t)syi * a.snyP + j;
        val = a.omega / a.c[J * a.NXg + I];
      }
      a.kedge[(int64_t)l * 4 * a.NE + k] = val;
    }
  }
}

// ---- b = (f, phi) + <g, phi>, lumped GLL quadrature (Sec. 4)
__global__ void rhs_kernel(const __grid_constant__ GlobalArgs a, const double* __restrict__ f,
                           const double* __restrict__ gb, double* __restrict__ b) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  if (I >= a.NXg) return;
  const int64_t n = (int64_t)J * a.NXg + I;
  const double wx = a.Wxg[I], wy = a.Wyg[J];
  double br = wx * wy * f[2 * n], bi = wx * wy * f[2 * n + 1];
  const int64_t oS = 0, oE = a.NXg, oN = a.NXg + a.NYg, oW = 2 * a.NXg + a.NYg;
  if (J == 0) { br += wx * gb[2 * (oS + I)]; bi += wx * gb[2 * (oS + I) + 1]; }
  if (J == a.NYg - 1) { br += wx * gb[2 * (oN + I)]; bi += wx * gb[2 * (oN + I) + 1]; }
  if (I == 0) { br += wy * gb[2 * (oW + J)]; bi += wy * gb[2 * (oW + J) + 1]; }
  if (I == a.NXg - 1) { br += wy * gb[2 * (oE + J)]; bi += wy * gb[2 * (oE + J) + 1]; }
  b[2 * n] = br;
  b[2 * n + 1] = bi;
}

// ---- r = b - (A - i w H - w^2 M) u on the global grid (Sec. 4), FP64.
// A u = Wy_J (Kx u)_IJ + Wx_I (Ky u)_IJ with assembled 1D rows built from the
// reference element stiffness (one-sided at the outer boundary).
template <int P>
__global__ void residual_kernel(const __grid_constant__ GlobalArgs a, const double* __restrict__ b,
                                const double* __restrict__ u, double* __restrict__ r, double* __restrict__ part) {
  // the assembled rows in shared memory: the lanes of a warp index them by
  // their own node class (a per-lane index into parameter space serialises)
  __shared__ double kx[P + 2][2 * P + 1], ky[P + 2][2 * P + 1];
  for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < (P + 2) * (2 * P + 1); k += blockDim.x * blockDim.y) {
    kx[k / (2 * P + 1)][k % (2 * P + 1)] = a.Kx[k / (2 * P + 1)][k % (2 * P + 1)];
    ky[k / (2 * P + 1)][k % (2 * P + 1)] = a.Ky[k / (2 * P + 1)][k % (2 * P + 1)];
  }
  __syncthreads();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  double sums[2] = {0.0, 0.0};
  if (I < a.NXg && J < a.NYg) {
    const int64_t n = (int64_t)J * a.NXg + I;
    const double2* u2 = reinterpret_cast<const double2*>(u);
    // x and y: assembled rows from the host tables (node class by position
    // in its element, first and last node of the mesh separately)
    const int cx = (I == 0) ? P : (I == a.NXg - 1) ? P + 1 : I % P;
    const int cy = (J == 0) ? P : (J == a.NYg - 1) ? P + 1 : J % P;
    double sxr = 0.0, sxi = 0.0, syr = 0.0, syi = 0.0;
#pragma unroll
    for (int tt = -P; tt <= P; ++tt) {
      if (I + tt >= 0 && I + tt < a.NXg) {  // taps outside the mesh have coefficient 0
        const double2 v = __ldg(&u2[n + tt]);
        const double cf = kx[cx][tt + P];
        sxr = fma(cf, v.x, sxr);
        sxi = fma(cf, v.y, sxi);
      }
      if (J + tt >= 0 && J + tt < a.NYg) {
        const double2 v = __ldg(&u2[n + (int64_t)tt * a.NXg]);
        const double cf = ky[cy][tt + P];
        syr = fma(cf, v.x, syr);
        syi = fma(cf, v.y, syi);
      }
    }
    const double Wx = a.Wxg[I], Wy = a.Wyg[J];
    const double Aur = Wy * sxr + Wx * syr;
    const double Aui = Wy * sxi + Wx * syi;
    const double c = a.c[n];
    const double M = Wx * Wy / (c * c);
    const double H = (((J == 0 || J == a.NYg - 1) ? Wx : 0.0) + ((I == 0 || I == a.NXg - 1) ? Wy : 0.0)) / c;
    const double2 un = u2[n];
    const double w = a.omega;
    // K u = A u - i w H u - w^2 M u
    const double Kur = Aur + w * H * un.y - w * w * M * un.x;
    const double Kui = Aui - w * H * un.x - w * w * M * un.y;
    double br = 0.0, bi = 0.0;
    if (b) { br = b[2 * n]; bi = b[2 * n + 1]; }
    const double rr = br - Kur, ri = bi - Kui;
    r[2 * n] = rr;
    r[2 * n + 1] = ri;
    sums[0] = rr * rr + ri * ri;
    sums[1] = br * br + bi * bi;
  }
  // flatten the 2D block for the reduction
  __shared__ double out[2];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  {
    __shared__ double sh[2][32];
    const int lane = tid & 31, warp = tid >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int k = 0; k < 2; ++k) {
      double x = warp_sum(sums[k]);
      if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
      for (int k = 0; k < 2; ++k) {
        double x = (lane < nw) ? sh[k][lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) out[k] = x;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * blk] = out[0];
    part[2 * blk + 1] = out[1];
  }
}

// out[k] = sum_blk part[blk * width + k], fixed order; one block per k.
__global__ void reduce_partials_kernel(const double* __restrict__ part, int nblocks, int width,
                                       double* __restrict__ out) {
  const int k = blockIdx.x;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v[0] += part[(int64_t)b * width + k];
  __shared__ double res[1];
  block_sum<1>(v, res);
  if (threadIdx.x == 0) out[k] = res[0];
}

// u += average of the subdomain copies at every global node, weighted by the
// lumped-mass share of each copy (1/count on a uniform mesh: 1, 1/2 on
// interfaces, 1/4 at cross points; a.share on a mapped mesh).
__global__ void assemble_add_kernel(const __grid_constant__ AssembleArgs a, const double* __restrict__ u_sub,
                                    double* __restrict__ u) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  if (I >= a.NXg) return;
  int sx1 = I / a.snxP, sx0 = sx1;
  if (sx1 >= a.Sx) { sx1 = a.Sx - 1; sx0 = sx1; }
  else if (I % a.snxP == 0 && I > 0) sx0 = sx1 - 1;
  int sy1 = J / a.snyP, sy0 = sy1;
  if (sy1 >= a.Sy) { sy1 = a.Sy - 1; sy0 = sy1; }
  else if (J % a.snyP == 0 && J > 0) sy0 = sy1 - 1;
  const double uniform = 1.0 / (double)((sx1 - sx0 + 1) * (sy1 - sy0 + 1));
  const int64_t nn = (int64_t)a.nlx * a.nly;
  double sr = 0.0, si = 0.0;
  for (int sy = sy0; sy <= sy1; ++sy)
    for (int sx = sx0; sx <= sx1; ++sx) {
      const int l = sy * a.Sx + sx;
      const int i = I - sx * a.snxP, j = J - sy * a.snyP;
      const int64_t k = (int64_t)l * nn + (int64_t)j * a.nlx + i;
      const double sh = a.share ? a.share[k] : 1.0;
      sr += sh * u_sub[2 * k];
      si += sh * u_sub[2 * k + 1];
    }
  const double scale = a.share ? 1.0 : uniform;
  const int64_t n = (int64_t)J * a.NXg + I;
  u[2 * n] += scale * sr;
  u[2 * n + 1] += scale * si;
}

// ---- Krylov vector kernels (vectors of n2 doubles = n2/2 complex values)
// On this part FP64 arithmetic, not memory, bounds these kernels (the FP64
// pipe retires about 1/65 of the FP32 rate), so they are written for the
// fewest FP64 instructions: every complex multiply-accumulate is four fma()
// (no separate multiply and add), the real variants skip the imaginary half,
// and the difference w = v - S v and the final norm ride along with the dot
// and update passes instead of running as passes of their own.
//
// multi_dot: one block per contiguous chunk of the vectors: the chunk of w is
// staged in shared memory once, then the block's warps take the basis vectors
// in turn (coalesced reads of each V_k chunk, two accumulator pairs per lane,
// one warp reduction per vector), so every element of V and w is read from
// memory once per call.  part[(blk * nv + k) * 2 + {0, 1}].
constexpr int kDotWarps = 8;
template <bool REAL, bool DIFF>
__global__ void __launch_bounds__(kDotWarps * 32)
    multi_dot_kernel(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w,
                     const double* __restrict__ w_sub, double* __restrict__ w_out, int64_t nc, int chunk,
                     double* __restrict__ part) {
  extern __shared__ double2 ws[];
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int rows = (int)((nc - r0) < chunk ? (nc - r0) : chunk);
  for (int q = threadIdx.x; q < rows; q += blockDim.x) {
    double2 x = reinterpret_cast<const double2*>(w)[r0 + q];
    if (DIFF) {
      const double2 y = reinterpret_cast<const double2*>(w_sub)[r0 + q];
      x.x -= y.x;
      x.y -= y.y;
      reinterpret_cast<double2*>(w_out)[r0 + q] = x;
    }
    ws[q] = x;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < nv; k += kDotWarps) {
    const double2* vk = reinterpret_cast<const double2*>(V + (int64_t)k * ld) + r0;
    // conj(a) b = (a.x b.x + a.y b.y) + i (a.x b.y - a.y b.x)
    double sr0 = 0.0, si0 = 0.0, sr1 = 0.0, si1 = 0.0;
    int q = lane;
#pragma unroll 2
    for (; q + 32 < rows; q += 64) {
      const double2 a = vk[q], b = ws[q], c = vk[q + 32], d = ws[q + 32];
      sr0 = fma(a.x, b.x, sr0);
      sr0 = fma(a.y, b.y, sr0);
      sr1 = fma(c.x, d.x, sr1);
      sr1 = fma(c.y, d.y, sr1);
      if (!REAL) {
        si0 = fma(a.x, b.y, si0);
        si0 = fma(-a.y, b.x, si0);
        si1 = fma(c.x, d.y, si1);
        si1 = fma(-c.y, d.x, si1);
      }
    }
    if (q < rows) {
      const double2 a = vk[q], b = ws[q];
      sr0 = fma(a.x, b.x, sr0);
      sr0 = fma(a.y, b.y, sr0);
      if (!REAL) {
        si0 = fma(a.x, b.y, si0);
        si0 = fma(-a.y, b.x, si0);
      }
    }
    const double sr = warp_sum(sr0 + sr1);
    const double si = REAL ? 0.0 : warp_sum(si0 + si1);
    if (lane == 0) {
      double* p = part + ((int64_t)blockIdx.x * nv + k) * 2;
      p[0] = sr;
      p[1] = si;
    }
  }
}

// w -= sum_k h_k V_k, one complex entry per thread and iteration, basis
// vectors taken two at a time into separate accumulators; NORM: the block's
// partial ||w_new||^2 into norm_part[2 blk] (0 into norm_part[2 blk + 1]).
template <bool REAL, bool NORM>
__global__ void multi_axpy_kernel(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ h,
                                  double* __restrict__ w, int64_t nc, double* __restrict__ norm_part) {
  extern __shared__ double hs[];
  for (int k = threadIdx.x; k < 2 * nv; k += blockDim.x) hs[k] = h[k];
  __syncthreads();
  double2* w2 = reinterpret_cast<double2*>(w);
  double nrm[1] = {0.0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nc; q += (int64_t)gridDim.x * blockDim.x) {
    // (hr + i hi)(v.x + i v.y) = (hr v.x - hi v.y) + i (hr v.y + hi v.x)
    double2 acc = w2[q], acc1 = make_double2(0.0, 0.0);
    int k = 0;
#pragma unroll 2
    for (; k + 1 < nv; k += 2) {
      const double2 v = reinterpret_cast<const double2*>(V + (int64_t)k * ld)[q];
      const double2 u = reinterpret_cast<const double2*>(V + (int64_t)(k + 1) * ld)[q];
      const double hr = hs[2 * k], hr1 = hs[2 * k + 2];
      acc.x = fma(-hr, v.x, acc.x);
      acc.y = fma(-hr, v.y, acc.y);
      acc1.x = fma(-hr1, u.x, acc1.x);
      acc1.y = fma(-hr1, u.y, acc1.y);
      if (!REAL) {
        const double hi = hs[2 * k + 1], hi1 = hs[2 * k + 3];
        acc.x = fma(hi, v.y, acc.x);
        acc.y = fma(-hi, v.x, acc.y);
        acc1.x = fma(hi1, u.y, acc1.x);
        acc1.y = fma(-hi1, u.x, acc1.y);
      }
    }
    if (k < nv) {
      const double2 v = reinterpret_cast<const double2*>(V + (int64_t)k * ld)[q];
      const double hr = hs[2 * k];
      acc.x = fma(-hr, v.x, acc.x);
      acc.y = fma(-hr, v.y, acc.y);
      if (!REAL) {
        const double hi = hs[2 * k + 1];
        acc.x = fma(hi, v.y, acc.x);
        acc.y = fma(-hi, v.x, acc.y);
      }
    }
    acc.x += acc1.x;
    acc.y += acc1.y;
    w2[q] = acc;
    if (NORM) nrm[0] = fma(acc.x, acc.x, fma(acc.y, acc.y, nrm[0]));
  }
  if (NORM) {
    __shared__ double res[1];
    block_sum<1>(nrm, res);
    if (threadIdx.x == 0) {
      norm_part[2 * blockIdx.x] = res[0];
      norm_part[2 * blockIdx.x + 1] = 0.0;
    }
  }
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n2) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = a * x[q] + b * y[q];
}

// y = x / sqrt(n2[0]) (0 if the norm is 0): normalises the next Krylov vector
// on the device, without a round trip to the host (y may be x).  With flags_src
// the solve's 4 status words are staged beside the Hessenberg column, so one
// device-to-host copy carries both.
__global__ void scale_inv_norm_kernel(const double* x, const double* __restrict__ n2, double* y, int64_t n,
                                      const int* __restrict__ flags_src, int* __restrict__ flags_dst) {
  if (flags_src && blockIdx.x == 0 && threadIdx.x < 4) flags_dst[threadIdx.x] = flags_src[threadIdx.x];
  const double v = n2[0];
  const double s = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    y[q] = s * x[q];
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * 8;  // 8 resident blocks of 256 threads per SM
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <int P>
hz_status launch_residual_P(const GlobalArgs& a, const double* b, const double* u, double* r, double* part,
                            int* nb, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((a.NXg + 31) / 32, (a.NYg + 7) / 8);
  residual_kernel<P><<<grd, blk, 0, st>>>(a, b, u, r, part);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  *nb = (int)(grd.x * grd.y);
  return HZ_OK;
}

}  // namespace

hz_status launch_prepare(const PrepArgs& a, int L, cudaStream_t st) {
  const int nn = a.nlx * a.nly;
  dim3 grd((nn + 255) / 256, L);
  prepare_kernel<<<grd, 256, 0, st>>>(a);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_rhs(const GlobalArgs& a, const double* f, const double* gb, double* b, cudaStream_t st) {
  dim3 grd((a.NXg + 127) / 128, a.NYg);
  rhs_kernel<<<grd, 128, 0, st>>>(a, f, gb, b);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

int residual_blocks(const GlobalArgs& a) { return ((a.NXg + 31) / 32) * ((a.NYg + 7) / 8); }

hz_status launch_residual(const GlobalArgs& a, const double* b, const double* u, double* r, double* part,
                          int* nblocks, cudaStream_t st) {
  switch (a.P) {
    case 1: return launch_residual_P<1>(a, b, u, r, part, nblocks, st);
    case 2: return launch_residual_P<2>(a, b, u, r, part, nblocks, st);
    case 3: return launch_residual_P<3>(a, b, u, r, part, nblocks, st);
    case 4: return launch_residual_P<4>(a, b, u, r, part, nblocks, st);
    case 5: return launch_residual_P<5>(a, b, u, r, part, nblocks, st);
    case 6: return launch_residual_P<6>(a, b, u, r, part, nblocks, st);
    case 7: return launch_residual_P<7>(a, b, u, r, part, nblocks, st);
    default: return fail(HZ_ERR_UNSUPPORTED, "degree outside 1..7");
  }
}

hz_status launch_reduce_partials(const double* part, int nblocks, int width, double* out, cudaStream_t st) {
  reduce_partials_kernel<<<width, kRedThreads, 0, st>>>(part, nblocks, width, out);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_assemble_add(const AssembleArgs& a, const double* u_sub, double* u, cudaStream_t st) {
  dim3 grd((a.NXg + 127) / 128, a.NYg);
  assemble_add_kernel<<<grd, 128, 0, st>>>(a, u_sub, u);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];  // 0 = not looked up yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    (void)cudaGetLastError();
    return 1;  // grid-stride kernels stay correct with any grid
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    (void)cudaGetLastError();
    v = 1;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// blocks for multi_dot: 2 per SM, chunks of at most 4096 complex entries (64 KB of shared memory)
int vec_blocks(int64_t n2) {
  const int64_t nc = n2 / 2;
  int64_t nb = 2 * (int64_t)sm_count();
  if ((nc + nb - 1) / nb > 4096) nb = (nc + 4095) / 4096;
  if (nb > nc) nb = nc > 0 ? nc : 1;
  return (int)nb;
}

template <bool REAL, bool DIFF>
hz_status launch_multi_dot_T(const double* V, int64_t ld, int nv, const double* w, const double* w_sub, double* w_out,
                             int64_t nc, int chunk, size_t smem, double* part, int nblocks, cudaStream_t st) {
  if (smem > 48 * 1024)
    HZ_CUDA(cudaFuncSetAttribute(multi_dot_kernel<REAL, DIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  multi_dot_kernel<REAL, DIFF><<<nblocks, kDotWarps * 32, smem, st>>>(V, ld, nv, w, w_sub, w_out, nc, chunk, part);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, const double* w_sub, double* w_out,
                           int64_t n2, bool real_dot, double* part, int nblocks, cudaStream_t st) {
  if ((w_sub == nullptr) != (w_out == nullptr)) return fail(HZ_ERR_INVALID_ARG, "multi_dot: w_sub and w_out go together");
  const int64_t nc = n2 / 2;
  const int chunk = (int)((nc + nblocks - 1) / nblocks);
  const size_t smem = (size_t)chunk * sizeof(double2);
  if (real_dot)
    return w_sub ? launch_multi_dot_T<true, true>(V, ld, nv, w, w_sub, w_out, nc, chunk, smem, part, nblocks, st)
                 : launch_multi_dot_T<true, false>(V, ld, nv, w, w_sub, w_out, nc, chunk, smem, part, nblocks, st);
  return w_sub ? launch_multi_dot_T<false, true>(V, ld, nv, w, w_sub, w_out, nc, chunk, smem, part, nblocks, st)
               : launch_multi_dot_T<false, false>(V, ld, nv, w, w_sub, w_out, nc, chunk, smem, part, nblocks, st);
}

int axpy_blocks(int64_t n2) { return grid_for(n2 / 2, 256); }

hz_status launch_multi_axpy(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n2,
                            bool real_coef, cudaStream_t st, double* norm_part) {
  const int64_t nc = n2 / 2;
  const int g = axpy_blocks(n2);
  const size_t smem = (size_t)2 * nv * sizeof(double);
  if (smem > 48 * 1024) {
    // nv above 3072 basis vectors: not reachable with the restart bound, refuse rather than launch
    return fail(HZ_ERR_UNSUPPORTED, "multi_axpy: too many basis vectors");
  }
  if (real_coef) {
    if (norm_part) multi_axpy_kernel<true, true><<<g, 256, smem, st>>>(V, ld, nv, h, w, nc, norm_part);
    else multi_axpy_kernel<true, false><<<g, 256, smem, st>>>(V, ld, nv, h, w, nc, nullptr);
  } else {
    if (norm_part) multi_axpy_kernel<false, true><<<g, 256, smem, st>>>(V, ld, nv, h, w, nc, norm_part);
    else multi_axpy_kernel<false, false><<<g, 256, smem, st>>>(V, ld, nv, h, w, nc, nullptr);
  }
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_scale_inv_norm(const double* x, const double* norm2, double* y, int64_t n2, cudaStream_t st,
                                const int* flags_src, int* flags_dst) {
  scale_inv_norm_kernel<<<grid_for(n2, 256), 256, 0, st>>>(x, norm2, y, n2, flags_src, flags_dst);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

// One thread per complex entry of the listed slots; slot k occupies entries
// [k NE, (k+1) NE) of the packed buffer.  A slot (l, e) outside the lambda
// vector (l not in 0..L-1 or e not in 0..3) is skipped: gather writes zeros
// for it, scatter writes nothing.
__global__ void lambda_slots_kernel(const int32_t* __restrict__ slots, int count, int NE, int L, const double2* src,
                                    double2* dst, int gather) {
  const int64_t total = (int64_t)count * NE;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / NE), t = (int)(q % NE);
    const int l = slots[2 * k], e = slots[2 * k + 1];
    const bool ok = l >= 0 && l < L && e >= 0 && e < 4;
    const int64_t slot = ((int64_t)l * 4 + e) * NE + t;
    if (gather) dst[q] = ok ? src[slot] : make_double2(0.0, 0.0);
    else if (ok) dst[slot] = src[q];
  }
}

hz_status launch_lambda_slots(const int32_t* slots, int count, int NE, int L, const double* src, double* dst,
                              bool gather, cudaStream_t st) {
  const int64_t total = (int64_t)count * NE;
  lambda_slots_kernel<<<grid_for(total, 256), 256, 0, st>>>(slots, count, NE, L, reinterpret_cast<const double2*>(src),
                                                             reinterpret_cast<double2*>(dst), gather ? 1 : 0);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_axpby(double a, const double* x, double b, double* y, int64_t n2, cudaStream_t st) {
  axpby_kernel<<<grid_for(n2, 256), 256, 0, st>>>(a, x, b, y, n2);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
