// Global residual without any device allocation.
//
// Some callers cannot allocate device memory: code running inside a CUDA
// graph being captured by someone else, a host process whose allocator is
// owned by another runtime (a game engine, a simulation framework with a
// fixed memory pool), or a real-time loop where cudaMalloc's implicit
// synchronisation is not allowed.  hz_residual_noalloc serves them: it
// computes the same r = b - K u and squared norms as hz_residual, from
// device arrays the caller owns, and keeps its block partial sums in a
// fixed-size array in this library's global memory (a file-scope
// __device__ array) instead of a library-allocated buffer.
//
// The array is a host-side stand-in in host code, not a device address: the
// host looks its device address up with cudaGetSymbolAddress, once per device
// (with that device current), and passes that address to the kernels.
// Every call shares the array; it keeps the last call's partial sums (each
// call overwrites every entry it reads, so nothing needs clearing), and calls
// that overlap on the GPU (different streams, same device) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hz_internal.h"

namespace hz {
namespace {

// Block partials: two doubles (|r|^2, |b|^2) per block of 32 x 8 nodes.
constexpr int kNoallocMaxBlocks = 1 << 17;  // meshes up to ~33.5 M nodes (2 MiB of scratch)
static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

hz_status scratch_for_current_device(double** out) {
  int dev = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HZ_ERR_UNSUPPORTED, "device index beyond the supported range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return HZ_OK;
}

}  // namespace
}  // namespace hz

namespace hz {
namespace {

struct NoallocArgs {
  int NXg, NYg, nx, ny;
  double omega, kxs, kys, hx2, hy2;
  double Kref[(kMaxP + 1) * (kMaxP + 1)];
  double w[kMaxP + 1];
};

__device__ __forceinline__ double warp_sum_na(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = b - (A - i w H - w^2 M) u (Sec. 4), the lumped 1D weights formed on the
// fly from the GLL weights (same products and summation order as the host
// tables of hz_residual); per-block partial sums into the static scratch.
template <int P>
__global__ void residual_noalloc_kernel(const __grid_constant__ NoallocArgs a, const double* __restrict__ c,
                                        const double* __restrict__ b, const double* __restrict__ u,
                                        double* __restrict__ r, double* __restrict__ part) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  double s0 = 0.0, s1 = 0.0;
  if (I < a.NXg && J < a.NYg) {
    const int64_t n = (int64_t)J * a.NXg + I;
    const double2* u2 = reinterpret_cast<const double2*>(u);
    const int ax = I % P, ex = I / P;
    const bool own_x = ex < a.nx, left_x = (ax == 0) && ex >= 1;
    double sxr = 0.0, sxi = 0.0;
#pragma unroll
    for (int tt = -P; tt <= P; ++tt) {
      double cf = 0.0;
      const int bb = ax + tt;
      const bool in_own = own_x && bb >= 0 && bb <= P, in_left = left_x && tt <= 0;
      if (in_own) cf += a.Kref[ax * (P + 1) + bb];
      if (in_left) cf += a.Kref[P * (P + 1) + (tt + P)];
      if (in_own || in_left) {
        const double2 v = __ldg(&u2[n + tt]);
        sxr += cf * v.x;
        sxi += cf * v.y;
      }
    }
    const int ay = J % P, ey = J / P;
    const bool own_y = ey < a.ny, below_y = (ay == 0) && ey >= 1;
    double syr = 0.0, syi = 0.0;
#pragma unroll
    for (int tt = -P; tt <= P; ++tt) {
      double cf = 0.0;
      const int bb = ay + tt;
      const bool in_own = own_y && bb >= 0 && bb <= P, in_below = below_y && tt <= 0;
      if (in_own) cf += a.Kref[ay * (P + 1) + bb];
      if (in_below) cf += a.Kref[P * (P + 1) + (tt + P)];
      if (in_own || in_below) {
        const double2 v = __ldg(&u2[n + (int64_t)tt * a.NXg]);
        syr += cf * v.x;
        syi += cf * v.y;
      }
    }
    const double Wx = (left_x ? a.w[P] * a.hx2 : 0.0) + (own_x ? a.w[ax] * a.hx2 : 0.0);
    const double Wy = (below_y ? a.w[P] * a.hy2 : 0.0) + (own_y ? a.w[ay] * a.hy2 : 0.0);
    const double Aur = Wy * a.kxs * sxr + Wx * a.kys * syr;
    const double Aui = Wy * a.kxs * sxi + Wx * a.kys * syi;
    const double cc = c[n];
    const double M = Wx * Wy / (cc * cc);
    const double H = (((J == 0 || J == a.NYg - 1) ? Wx : 0.0) + ((I == 0 || I == a.NXg - 1) ? Wy : 0.0)) / cc;
    const double2 un = u2[n];
    const double w = a.omega;
    const double Kur = Aur + w * H * un.y - w * w * M * un.x;
    const double Kui = Aui - w * H * un.x - w * w * M * un.y;
    double br = 0.0, bi = 0.0;
    if (b) { br = b[2 * n]; bi = b[2 * n + 1]; }
    const double rr = br - Kur, ri = bi - Kui;
    r[2 * n] = rr;
    r[2 * n + 1] = ri;
    s0 = rr * rr + ri * ri;
    s1 = br * br + bi * bi;
  }
  __shared__ double sh[2][32];
  __shared__ double out[2];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  double x0 = warp_sum_na(s0), x1 = warp_sum_na(s1);
  if (lane == 0) { sh[0][warp] = x0; sh[1][warp] = x1; }
  __syncthreads();
  if (warp == 0) {
    double y0 = (lane < nw) ? sh[0][lane] : 0.0, y1 = (lane < nw) ? sh[1][lane] : 0.0;
    y0 = warp_sum_na(y0);
    y1 = warp_sum_na(y1);
    if (lane == 0) { out[0] = y0; out[1] = y1; }
  }
  __syncthreads();
  if (tid == 0) {
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * blk] = out[0];
    part[2 * blk + 1] = out[1];
  }
}

template <int P>
void launch_na(const NoallocArgs& a, dim3 grd, const double* c, const double* b, const double* u, double* r,
               double* part, cudaStream_t st) {
  residual_noalloc_kernel<P><<<grd, dim3(32, 8), 0, st>>>(a, c, b, u, r, part);
}

}  // namespace
}  // namespace hz

using namespace hz;

extern "C" hz_status hz_residual_noalloc(hz_mesh mesh, double omega, const double* c, const double* b,
                                          const double* u, double* r, double* norms2, void* stream) {
  if (!mesh || !c || !u || !r || !norms2) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (!(omega > 0.0)) return fail(HZ_ERR_INVALID_ARG, "omega must be > 0");
  const Geom& g = mesh->g;
  const dim3 grd((g.NXg + 31) / 32, (g.NYg + 7) / 8);
  const int64_t nblocks = (int64_t)grd.x * grd.y;
  if (nblocks > kNoallocMaxBlocks)
    return fail(HZ_ERR_UNSUPPORTED, "mesh too large for hz_residual_noalloc: at most " +
                                        std::to_string((long long)kNoallocMaxBlocks) +
                                        " blocks of 32 x 8 nodes (about 33.5 M nodes)");
  if (grd.y > 65535u)  // the launch's y dimension: thin meshes with many node rows
    return fail(HZ_ERR_UNSUPPORTED, "mesh too large for hz_residual_noalloc: at most 65535 blocks of 8 node rows "
                                    "(524280 node rows)");
  double* part = nullptr;
  HZ_TRY(scratch_for_current_device(&part));
  NoallocArgs a{};
  a.NXg = g.NXg;
  a.NYg = g.NYg;
  a.nx = g.nx;
  a.ny = g.ny;
  a.omega = omega;
  a.kxs = 2.0 / g.hx;
  a.kys = 2.0 / g.hy;
  a.hx2 = g.hx / 2.0;
  a.hy2 = g.hy / 2.0;
  for (size_t k = 0; k < g.Kref.size(); ++k) a.Kref[k] = g.Kref[k];
  for (int k = 0; k <= g.P; ++k) a.w[k] = g.w[k];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (g.P) {
    case 1: launch_na<1>(a, grd, c, b, u, r, part, st); break;
    case 2: launch_na<2>(a, grd, c, b, u, r, part, st); break;
    case 3: launch_na<3>(a, grd, c, b, u, r, part, st); break;
    case 4: launch_na<4>(a, grd, c, b, u, r, part, st); break;
    case 5: launch_na<5>(a, grd, c, b, u, r, part, st); break;
    case 6: launch_na<6>(a, grd, c, b, u, r, part, st); break;
    case 7: launch_na<7>(a, grd, c, b, u, r, part, st); break;
    default: return fail(HZ_ERR_UNSUPPORTED, "degree outside 1..7");
  }
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return launch_reduce_partials(part, (int)nblocks, 2, norms2, st);
}
