// Register-resident sweep instantiations for degree 3: one warp per
// subdomain (h = 1) and, for the larger shapes, h = 2 or 4 warps per
// subdomain (row bands).
#include "hz_sweep_warp_launch.cuh"

namespace hz {
namespace warp_sweep {
hz_status launch_p3(int sy, int h, const WarpSweepArgs& a, cudaStream_t st) {
  switch (sy) {
    case 1: if (h == 1) return launch<3, 1, 1>(a, st); return HZ_ERR_UNSUPPORTED;
    case 2: if (h == 1) return launch<3, 2, 1>(a, st); return HZ_ERR_UNSUPPORTED;
    case 4: if (h == 1) return launch<3, 4, 1>(a, st); if (h == 2) return launch<3, 4, 2>(a, st); return HZ_ERR_UNSUPPORTED;
    case 8: if (h == 1) return launch<3, 8, 1>(a, st); if (h == 2) return launch<3, 8, 2>(a, st); if (h == 4) return launch<3, 8, 4>(a, st); return HZ_ERR_UNSUPPORTED;
    default: return HZ_ERR_UNSUPPORTED;
  }
}
}  // namespace warp_sweep
}  // namespace hz
