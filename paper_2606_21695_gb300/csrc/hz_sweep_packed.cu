// Packed multi-problem sweep: one launch performs one DD sweep (Algorithm 1)
// for several independent problems at once (different meshes, degrees,
// frequencies and N_t), every subdomain of every problem swept by one warp
// with the register-resident body of hz_sweep_warp.cuh.
//
// The launch is persistent: a grid of (resident blocks per SM) x (SMs)
// one-warp blocks walks the items (problem, subdomain) of all problems, the
// problems in decreasing order of cost per subdomain (nodes x (N_t - 1) x
// WaveHoltz iterations), so the longest items start first; an item finds its
// problem by binary search in the running subdomain counts.  Per-problem
// parameters (with the compiled shape id) are read from a table in global
// memory; the y-stiffness coefficients are the compile-time tables every
// problem of a degree shares.
#include <cuda_runtime.h>

#include "hz_sweep_warp.cuh"

namespace hz {
namespace {

// Shapes (P, subdomain elements in y) compiled into the packed kernel; the
// subdomain must also have at most 32 node columns.  The largest (P = 3,
// 8 elements, 25 rows) sets the kernel's register count.
#define HZ_PACKED_SHAPES(X) \
  X(0, 1, 4)                \
  X(1, 1, 8)                \
  X(2, 1, 16)               \
  X(3, 2, 4)                \
  X(4, 2, 8)                \
  X(5, 3, 4)                \
  X(6, 3, 8)                \
  X(7, 4, 4)                \
  X(8, 5, 4)

constexpr int kPackedMaxRows = 25;

__global__ void __launch_bounds__(32) sweep_packed_kernel(const WarpSweepArgs* __restrict__ descs,
                                                           const int* __restrict__ offsets, int R) {
  __shared__ float4 ec[kPackedMaxRows][2];
  const int nitems = offsets[R];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    // the problem holding item it: offsets[d] <= it < offsets[d + 1]
    int lo = 0, hi = R - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (offsets[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const WarpSweepArgs& x = descs[lo];
    const int l = it - offsets[lo];
    switch (2 * x.shape + (x.base.rhs != nullptr ? 1 : 0)) {
#define HZ_CASE(ID, P, SY)                                                 \
  case 2 * ID: warp_sweep::warp_body<P, SY, false, false>(x, l, ec, nullptr); break; \
  case 2 * ID + 1: warp_sweep::warp_body<P, SY, true, false>(x, l, ec, nullptr); break;
      HZ_PACKED_SHAPES(HZ_CASE)
#undef HZ_CASE
      default: break;  // the host only packs compiled shapes
    }
    __syncwarp();  // the edge table is rewritten by the next item
  }
}

}  // namespace

int packed_shape_id(int P, int sny, int nlx) {
  if (nlx > 32) return -1;
#define HZ_ID(ID, PP, SY) \
  if (P == PP && sny == SY) return ID;
  HZ_PACKED_SHAPES(HZ_ID)
#undef HZ_ID
  return -1;
}

hz_status launch_sweep_packed(const WarpSweepArgs* descs, const int* offsets, int R, cudaStream_t st) {
  if (R <= 0) return HZ_OK;
  int dev = 0, sms = 0, per_sm = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_packed_kernel, 32, 0));
  if (per_sm < 1) per_sm = 1;
  sweep_packed_kernel<<<per_sm * sms, 32, 0, st>>>(descs, offsets, R);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
