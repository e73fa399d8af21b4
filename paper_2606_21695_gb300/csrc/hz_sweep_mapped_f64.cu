// FP64 instantiation of the mapped-mesh sweep (hz_sweep_mapped.cuh).
#include "hz_sweep_mapped.cuh"

namespace hz {
hz_status launch_sweep_mapped_f64(int P, const MappedSweepArgs& a, int L, cudaStream_t st) {
  return launch_mapped_T<double>(P, a, L, st);
}
}  // namespace hz
