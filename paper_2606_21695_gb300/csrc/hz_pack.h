// Sweep packer: gathers the sweeps that concurrent solves on one device
// request and issues them as one packed launch (hz_sweep_packed.cu).
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <mutex>
#include <string>
#include <vector>

#include "hz_internal.h"
#include "hz_problem.h"

namespace hz {

class Packer {
 public:
  explicit Packer(int device);
  ~Packer();
  Packer(const Packer&) = delete;
  Packer& operator=(const Packer&) = delete;

  // True when the problem's sweeps can run in the packed kernel under these
  // options (FP32 sweeps, fixed WaveHoltz count, a compiled shape).
  static bool packable(const Problem& pr, const hz_solve_opts& o);

  // A solve that will route its sweeps here joins before its first sweep and
  // leaves after its last; the packer waits for every member's request
  // (or a short timeout) before launching.
  void join();
  void leave();

  // Queues one sweep of pr (parameters x, already prepared) ordered after the
  // work enqueued so far on st, and returns once the packed launch holding it
  // has been issued; st then waits for that launch.
  hz_status submit(Problem& pr, const WarpSweepArgs& x, int shape, cudaStream_t st);

  uint64_t launches() const { return launches_; }

 private:
  struct Req {
    Problem* pr;
    WarpSweepArgs x;
    int shape;
    bool src;
    cudaStream_t st;
    bool launched = false;
    hz_status status = HZ_OK;
    std::string error;
  };
  hz_status launch_locked();
  hz_status launch_batch(std::vector<Req*>& batch);

  int device_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::vector<Req*> pending_;
  int members_ = 0;
  long wait_us_;
  cudaStream_t st_ = nullptr;
  cudaEvent_t done_ = nullptr;
  // descriptor + running-count ring (pinned host staging -> device), one event per slot
  static constexpr int kRing = 4;
  HostBuf hdesc_[kRing];
  DevBuf ddesc_[kRing];
  cudaEvent_t ring_ev_[kRing] = {};
  int ring_ = 0;
  uint64_t launches_ = 0;
};

}  // namespace hz
