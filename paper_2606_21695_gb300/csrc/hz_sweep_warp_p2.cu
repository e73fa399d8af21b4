// Warp-per-subdomain sweep instantiations for degree 2.
#include "hz_sweep_warp.cuh"

namespace hz {
namespace warp_sweep {
namespace {
template <int P, int SY>
hz_status launch(const WarpSweepArgs& a, cudaStream_t st) {
  const int blocks = (a.L + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (a.base.rhs) sweep_warp_kernel<P, SY, true><<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
  else sweep_warp_kernel<P, SY, false><<<blocks, kWarpsPerBlock * 32, 0, st>>>(a);
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}
}  // namespace

hz_status launch_p2(int sy, const WarpSweepArgs& a, cudaStream_t st) {
  switch (sy) {
    case 1: return launch<2, 1>(a, st);
    case 2: return launch<2, 2>(a, st);
    case 4: return launch<2, 4>(a, st);
    case 8: return launch<2, 8>(a, st);
    default: return HZ_ERR_UNSUPPORTED;
  }
}
}  // namespace warp_sweep
}  // namespace hz
