// Packed multi-problem sweep: one launch performs one DD sweep (Algorithm 1)
// for several independent problems at once (different meshes, degrees,
// frequencies and N_t), every subdomain of every problem swept by one warp
// with the register-resident body of hz_sweep_warp.cuh.
//
// The launch is persistent: a grid of at most (resident blocks per SM) x
// (SMs) one-warp blocks walks a list of work items {problem, subdomain,
// shape}, sorted by decreasing cost (subdomain nodes x (N_t - 1) x WaveHoltz
// iterations) so the longest items start first.  Per-problem parameters are
// read from a table in global memory; the y-stiffness coefficients are the
// compile-time tables every problem of a degree shares.
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
                                                           const int4* __restrict__ items, int nitems) {
  __shared__ float4 ec[kPackedMaxRows][2];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];  // {descriptor, subdomain, shape, with source}
    const WarpSweepArgs& x = descs[w.x];
    switch (2 * w.z + w.w) {
#define HZ_CASE(ID, P, SY)                                                 \
  case 2 * ID: warp_sweep::warp_body<P, SY, false, false>(x, w.y, ec, nullptr); break; \
  case 2 * ID + 1: warp_sweep::warp_body<P, SY, true, false>(x, w.y, ec, nullptr); break;
      HZ_PACKED_SHAPES(HZ_CASE)
#undef HZ_CASE
      default: break;  // the host only builds items for compiled shapes
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

hz_status launch_sweep_packed(const WarpSweepArgs* descs, const int4* items, int nitems, cudaStream_t st) {
  if (nitems <= 0) return HZ_OK;
  int dev = 0, sms = 0, per_sm = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HZ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_packed_kernel, 32, 0));
  if (per_sm < 1) per_sm = 1;
  const int grid = nitems < per_sm * sms ? nitems : per_sm * sms;
  sweep_packed_kernel<<<grid, 32, 0, st>>>(descs, items, nitems);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
