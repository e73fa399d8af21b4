// Launch of one compiled variant of the register-resident sweep: degree P,
// SY elements per subdomain in y, H warps per subdomain (1: one warp,
// hz_sweep_warp.cuh; 2 or 4: row bands, hz_sweep_band.cuh), one subdomain per
// block.  The per-degree files (hz_sweep_warp_p1.cu ... p7.cu) list which
// (SY, H) pairs each degree compiles; they are split by degree so that nvcc
// builds them in parallel.
#pragma once

#include "hz_sweep_band.cuh"
#include "hz_sweep_warp.cuh"

namespace hz {
namespace warp_sweep {
namespace {

template <int P, int SY, int H>
hz_status launch(const WarpSweepArgs& a, cudaStream_t st) {
  if constexpr (H == 1) {
    const int blocks = a.L;  // one subdomain (one warp) per block
    const bool rm = a.base.eta != 0.0;  // interface boundary mass present
    if (a.base.u0) {  // warm start (the boundary-mass terms kept: zero when eta = 0)
      if (a.base.rhs) sweep_warp_kernel<P, SY, true, true, true><<<blocks, 32, 0, st>>>(a);
      else sweep_warp_kernel<P, SY, false, true, true><<<blocks, 32, 0, st>>>(a);
    } else if (a.base.rhs) {
      if (rm) sweep_warp_kernel<P, SY, true, true><<<blocks, 32, 0, st>>>(a);
      else sweep_warp_kernel<P, SY, true, false><<<blocks, 32, 0, st>>>(a);
    } else {
      if (rm) sweep_warp_kernel<P, SY, false, true><<<blocks, 32, 0, st>>>(a);
      else sweep_warp_kernel<P, SY, false, false><<<blocks, 32, 0, st>>>(a);
    }
  } else {
    const int blocks = a.L;  // one subdomain (H warps) per block
    if (a.base.u0) {
      if (a.base.rhs) band_sweep::sweep_band_kernel<P, SY, true, H, true><<<blocks, H * 32, 0, st>>>(a);
      else band_sweep::sweep_band_kernel<P, SY, false, H, true><<<blocks, H * 32, 0, st>>>(a);
    } else if (a.base.rhs) band_sweep::sweep_band_kernel<P, SY, true, H><<<blocks, H * 32, 0, st>>>(a);
    else band_sweep::sweep_band_kernel<P, SY, false, H><<<blocks, H * 32, 0, st>>>(a);
  }
  note_launch();
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}
}  // namespace
}  // namespace warp_sweep
}  // namespace hz
