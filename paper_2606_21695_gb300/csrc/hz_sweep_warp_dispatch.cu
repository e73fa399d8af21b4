// Dispatch of the register-resident sweep over the compiled (P, sub_ny, warps
// per subdomain) variants.
#include "hz_internal.h"

namespace hz {
namespace warp_sweep {
hz_status launch_p1(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p2(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p3(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p4(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p5(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p6(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
hz_status launch_p7(int sy, int h, const WarpSweepArgs& a, cudaStream_t st);
}  // namespace warp_sweep

hz_status launch_sweep_warp(int P, int sy, int h, const WarpSweepArgs& a, cudaStream_t st) {
  if (a.base.nlx > 32 || a.base.nly > kWarpMaxRows) return HZ_ERR_UNSUPPORTED;
  if (h != 1 && h != 2 && h != 4) return HZ_ERR_UNSUPPORTED;
  switch (P) {
    case 1: return warp_sweep::launch_p1(sy, h, a, st);
    case 2: return warp_sweep::launch_p2(sy, h, a, st);
    case 3: return warp_sweep::launch_p3(sy, h, a, st);
    case 4: return warp_sweep::launch_p4(sy, h, a, st);
    case 5: return warp_sweep::launch_p5(sy, h, a, st);
    case 6: return warp_sweep::launch_p6(sy, h, a, st);
    case 7: return warp_sweep::launch_p7(sy, h, a, st);
    default: return HZ_ERR_UNSUPPORTED;
  }
}
}  // namespace hz
