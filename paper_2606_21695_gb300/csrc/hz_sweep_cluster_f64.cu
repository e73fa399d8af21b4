// FP64 instantiation of the cluster sweep (hz_sweep_cluster.cuh).
#include "hz_sweep_cluster.cuh"

namespace hz {
hz_status launch_sweep_cluster_f64(int P, const SweepArgs& a, int L, cudaStream_t st) {
  return cluster_sweep::launch_any<double>(P, a, L, st);
}
}  // namespace hz
