// FP32 instantiation of the cluster sweep (hz_sweep_cluster.cuh).
#include "hz_sweep_cluster.cuh"

namespace hz {
hz_status launch_sweep_cluster(int P, const SweepArgs& a, int L, cudaStream_t st) {
  return cluster_sweep::launch_any<float>(P, a, L, st);
}
}  // namespace hz
