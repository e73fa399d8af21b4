// FP64 global kernels for meshes of general convex quadrilaterals: the
// right-hand side b = (f, phi) + <g, phi> and the residual r = b - K u with
// K = A - i w H - w^2 M (Sec. 4), A in the element form with the map's metric
// (see hz_mapped.cpp), M and H lumped.  Both run once per refinement step;
// they are written for clarity: one thread per element node for the metric
// fluxes of u, one thread per global node for the assembly gather.
#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {
namespace {

__device__ __forceinline__ double warp_sum_m(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// b = W f + (arc-length weight) g on the outer edges (S, E, N, W order)
__global__ void rhs_mapped_kernel(const __grid_constant__ MappedGlobalArgs a, const double* __restrict__ f,
                                  const double* __restrict__ gb, double* __restrict__ b) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y;
  if (I >= a.NXg) return;
  const int64_t n = (int64_t)J * a.NXg + I;
  const double W = a.W[n];
  double br = W * f[2 * n], bi = W * f[2 * n + 1];
  const int64_t oS = 0, oE = a.NXg, oN = a.NXg + a.NYg, oW = 2 * a.NXg + a.NYg;
  auto add = [&](int64_t k) {
    br += a.bw[k] * gb[2 * k];
    bi += a.bw[k] * gb[2 * k + 1];
  };
  if (J == 0) add(oS + I);
  if (J == a.NYg - 1) add(oN + I);
  if (I == 0) add(oW + J);
  if (I == a.NXg - 1) add(oE + J);
  b[2 * n] = br;
  b[2 * n + 1] = bi;
}

// metric fluxes of u at every element node: flux[(e N2 + loc) 4 + {F1 re, F1 im, F2 re, F2 im}]
template <int P>
__global__ void flux_mapped_kernel(const __grid_constant__ MappedGlobalArgs a, const double* __restrict__ u) {
  constexpr int M = P + 1, N2 = M * M;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nel = (int64_t)a.nx * a.ny;
  if (idx >= nel * N2) return;
  const int64_t e = idx / N2;
  const int loc = (int)(idx - e * N2);
  const int b = loc / M, aa = loc - b * M;
  const int ex = (int)(e % a.nx), ey = (int)(e / a.nx);
  const double2* u2 = reinterpret_cast<const double2*>(u);
  const int64_t row0 = ((int64_t)ey * P + b) * a.NXg + (int64_t)ex * P;
  const int64_t col0 = ((int64_t)ey * P) * a.NXg + (int64_t)ex * P + aa;
  double xr = 0, xi = 0, er = 0, ei = 0;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    const double2 vr = u2[row0 + c];
    const double2 vc = u2[col0 + (int64_t)c * a.NXg];
    xr += a.D[aa * M + c] * vr.x;
    xi += a.D[aa * M + c] * vr.y;
    er += a.D[b * M + c] * vc.x;
    ei += a.D[b * M + c] * vc.y;
  }
  const double* g = a.geo + idx * 3;
  double* F = a.flux + idx * 4;
  F[0] = g[0] * xr + g[1] * er;
  F[1] = g[0] * xi + g[1] * ei;
  F[2] = g[1] * xr + g[2] * er;
  F[3] = g[1] * xi + g[2] * ei;
}

// A u at every global node by gathering D^T F from its (up to four) elements;
// r = b - (A u - i w H u - w^2 M u); per-block partial |r|^2, |b|^2.
template <int P>
__global__ void gather_mapped_kernel(const __grid_constant__ MappedGlobalArgs a, const double* __restrict__ b,
                                     const double* __restrict__ u, double* __restrict__ r,
                                     double* __restrict__ part) {
  constexpr int M = P + 1, N2 = M * M;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  double s0 = 0.0, s1 = 0.0;
  if (I < a.NXg && J < a.NYg) {
    int ex[2], ax[2], nex = 0, ey[2], by[2], ney = 0;
    if (I % P == 0 && I > 0) { ex[nex] = I / P - 1; ax[nex] = P; ++nex; }
    if (I / P < a.nx) { ex[nex] = I / P; ax[nex] = I % P; ++nex; }
    if (J % P == 0 && J > 0) { ey[ney] = J / P - 1; by[ney] = P; ++ney; }
    if (J / P < a.ny) { ey[ney] = J / P; by[ney] = J % P; ++ney; }
    double ar = 0.0, ai = 0.0;
    for (int qy = 0; qy < ney; ++qy)
      for (int qx = 0; qx < nex; ++qx) {
        const int64_t e = (int64_t)ey[qy] * a.nx + ex[qx];
        const int aa = ax[qx], bb = by[qy];
        const double* F = a.flux + e * N2 * 4;
#pragma unroll
        for (int q = 0; q < M; ++q) {
          const double d1 = a.D[q * M + aa], d2 = a.D[q * M + bb];
          const double* F1 = F + (bb * M + q) * 4;  // F1(bb, q)
          const double* F2 = F + (q * M + aa) * 4;  // F2(q, aa)
          ar += d1 * F1[0] + d2 * F2[2];
          ai += d1 * F1[1] + d2 * F2[3];
        }
      }
    const int64_t n = (int64_t)J * a.NXg + I;
    const double c = a.c[n];
    const double Mm = a.W[n] / (c * c), H = a.Hw[n] / c, w = a.omega;
    const double ur = u[2 * n], ui = u[2 * n + 1];
    // K u = A u - i w H u - w^2 M u
    const double kr = ar + w * H * ui - w * w * Mm * ur;
    const double ki = ai - w * H * ur - w * w * Mm * ui;
    const double br = b ? b[2 * n] : 0.0, bi = b ? b[2 * n + 1] : 0.0;
    const double rr = br - kr, ri = bi - ki;
    r[2 * n] = rr;
    r[2 * n + 1] = ri;
    s0 = rr * rr + ri * ri;
    s1 = br * br + bi * bi;
  }
  // block sums (fixed order)
  __shared__ double sh[2][32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
  s0 = warp_sum_m(s0);
  s1 = warp_sum_m(s1);
  if (lane == 0) {
    sh[0][warp] = s0;
    sh[1][warp] = s1;
  }
  __syncthreads();
  if (warp == 0) {
    double x0 = lane < nw ? sh[0][lane] : 0.0, x1 = lane < nw ? sh[1][lane] : 0.0;
    x0 = warp_sum_m(x0);
    x1 = warp_sum_m(x1);
    if (lane == 0) {
      const int blk = blockIdx.y * gridDim.x + blockIdx.x;
      part[2 * blk] = x0;
      part[2 * blk + 1] = x1;
    }
  }
}

template <int P>
hz_status residual_mapped_P(const MappedGlobalArgs& a, const double* b, const double* u, double* r, double* part,
                            int* nblocks, cudaStream_t st) {
  constexpr int N2 = (P + 1) * (P + 1);
  const int64_t total = (int64_t)a.nx * a.ny * N2;
  flux_mapped_kernel<P><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, u);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  dim3 blk(32, 8);
  dim3 grd((a.NXg + 31) / 32, (a.NYg + 7) / 8);
  gather_mapped_kernel<P><<<grd, blk, 0, st>>>(a, b, u, r, part);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  *nblocks = (int)(grd.x * grd.y);
  return HZ_OK;
}

}  // namespace

hz_status launch_rhs_mapped(const MappedGlobalArgs& a, const double* f, const double* gb, double* b,
                            cudaStream_t st) {
  dim3 grd((a.NXg + 127) / 128, a.NYg);
  rhs_mapped_kernel<<<grd, 128, 0, st>>>(a, f, gb, b);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

int residual_mapped_blocks(const MappedGlobalArgs& a) { return ((a.NXg + 31) / 32) * ((a.NYg + 7) / 8); }

hz_status launch_residual_mapped(const MappedGlobalArgs& a, const double* b, const double* u, double* r, double* part,
                                 int* nblocks, cudaStream_t st) {
  switch (a.P) {
    case 1: return residual_mapped_P<1>(a, b, u, r, part, nblocks, st);
    case 2: return residual_mapped_P<2>(a, b, u, r, part, nblocks, st);
    case 3: return residual_mapped_P<3>(a, b, u, r, part, nblocks, st);
    case 4: return residual_mapped_P<4>(a, b, u, r, part, nblocks, st);
    case 5: return residual_mapped_P<5>(a, b, u, r, part, nblocks, st);
    case 6: return residual_mapped_P<6>(a, b, u, r, part, nblocks, st);
    case 7: return residual_mapped_P<7>(a, b, u, r, part, nblocks, st);
    default: return fail(HZ_ERR_UNSUPPORTED, "degree outside 1..7");
  }
}

}  // namespace hz
