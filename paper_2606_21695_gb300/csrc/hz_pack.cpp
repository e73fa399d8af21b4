// Sweep packer (see hz_pack.h).
//
// Solves that run concurrently on one device (hz_solve_batch, the server)
// each drive their own outer iteration on their own stream.  Instead of one
// sweep launch per solve, every member hands its sweep request here; when all
// members have a request pending (or the oldest has waited wait_us), one
// thread issues a single packed launch covering all of them on the packer's
// stream, after each member's stream reached its request (events), and makes
// each member's stream wait for the launch.  The members' outer iterations
// thus advance in lockstep, one packed launch per step, and their vector
// kernels overlap on their own streams.
//
// A member's result does not depend on what else is in the pack: each
// subdomain is swept by one warp with the same arithmetic whatever its
// neighbours in the launch are.
#include "hz_pack.h"

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>

namespace hz {

Packer::Packer(int device) : device_(device) {
  const char* w = std::getenv("HZ_PACK_WAIT_US");
  wait_us_ = w ? std::max(1L, std::atol(w)) : 300L;
  cudaSetDevice(device_);
  cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&done_, cudaEventDisableTiming);
  for (int k = 0; k < kRing; ++k) cudaEventCreateWithFlags(&ring_ev_[k], cudaEventDisableTiming);
}

Packer::~Packer() {
  cudaSetDevice(device_);
  if (st_) cudaStreamSynchronize(st_);
  for (int k = 0; k < kRing; ++k)
    if (ring_ev_[k]) cudaEventDestroy(ring_ev_[k]);
  if (done_) cudaEventDestroy(done_);
  if (st_) cudaStreamDestroy(st_);
}

bool Packer::packable(const Problem& pr, const hz_solve_opts& o) {
  if (o.precision != HZ_FP32_REFINE || o.wh_tol > 0.0 || o.wh_adaptive || o.wh_warm || pr.mapped) return false;
  return packed_shape_id(pr.g.P, pr.g.sny, pr.g.nlx) >= 0;
}

void Packer::join() {
  std::lock_guard<std::mutex> lk(mu_);
  ++members_;
}

void Packer::leave() {
  std::unique_lock<std::mutex> lk(mu_);
  --members_;
  // the requests still pending may now be all there is to wait for
  if (!pending_.empty() && (int)pending_.size() >= members_) launch_locked();
}

hz_status Packer::submit(Problem& pr, const WarpSweepArgs& x, int shape, cudaStream_t st) {
  if (!pr.pack_ready) HZ_CUDA(cudaEventCreateWithFlags(&pr.pack_ready, cudaEventDisableTiming));
  HZ_CUDA(cudaEventRecord(pr.pack_ready, st));
  Req r{&pr, x, shape, x.base.rhs != nullptr, st};
  std::unique_lock<std::mutex> lk(mu_);
  pending_.push_back(&r);
  // Launch when every member has a request pending, or when the oldest
  // request has waited wait_us.  (Launching as soon as the previous packed
  // launch had finished was measured slower: smaller packs, more launches.)
  if ((int)pending_.size() >= members_) {
    launch_locked();
  } else {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(wait_us_);
    cv_.wait_until(lk, deadline, [&] { return r.launched; });
    if (!r.launched) launch_locked();  // timed out: launch what has gathered
  }
  if (r.status != HZ_OK) set_error(r.error);
  return r.status;
}

hz_status Packer::launch_locked() {
  std::vector<Req*> batch;
  batch.swap(pending_);
  hz_status s = launch_batch(batch);
  std::string msg;
  if (s != HZ_OK) {
    char buf[512] = {0};
    hz_last_error(buf, sizeof buf);
    msg = buf;
  }
  for (Req* r : batch) {
    r->status = s;
    r->error = msg;
    r->launched = true;
  }
  cv_.notify_all();
  return s;
}

hz_status Packer::launch_batch(std::vector<Req*>& batch) {
  if (batch.empty()) return HZ_OK;
  HZ_CUDA(cudaSetDevice(device_));
  // longest items first (cost per subdomain), ties by problem address for a
  // stable plan
  auto cost = [](const Req* r) {
    return (double)r->pr->g.sub_nodes() * (r->x.base.Nt - 1) * r->x.base.m_wh;
  };
  std::sort(batch.begin(), batch.end(), [&](const Req* a, const Req* b) {
    const double ca = cost(a), cb = cost(b);
    if (ca != cb) return ca > cb;
    return a->pr < b->pr;
  });
  const int R = (int)batch.size();
  // descriptors, then R + 1 running subdomain counts, into the next ring slot
  const int slot = ring_;
  ring_ = (ring_ + 1) % kRing;
  HZ_CUDA(cudaEventSynchronize(ring_ev_[slot]));  // its previous copy is done
  const size_t db = (size_t)R * sizeof(WarpSweepArgs);
  const size_t total = db + (size_t)(R + 1) * sizeof(int);
  if (total > ddesc_[slot].bytes) {
    HZ_CUDA(cudaStreamSynchronize(st_));
    HZ_TRY(ddesc_[slot].ensure(total));
  }
  HZ_TRY(hdesc_[slot].ensure(total));
  WarpSweepArgs* hd = hdesc_[slot].as<WarpSweepArgs>();
  int* off = reinterpret_cast<int*>(static_cast<char*>(hdesc_[slot].ptr) + db);
  off[0] = 0;
  for (int d = 0; d < R; ++d) {
    hd[d] = batch[d]->x;
    hd[d].shape = batch[d]->shape;
    off[d + 1] = off[d] + batch[d]->x.L;
  }
  for (const Req* r : batch) HZ_CUDA(cudaStreamWaitEvent(st_, r->pr->pack_ready, 0));
  HZ_CUDA(cudaMemcpyAsync(ddesc_[slot].ptr, hdesc_[slot].ptr, total, cudaMemcpyHostToDevice, st_));
  HZ_CUDA(cudaEventRecord(ring_ev_[slot], st_));
  HZ_TRY(launch_sweep_packed(ddesc_[slot].as<WarpSweepArgs>(),
                             reinterpret_cast<const int*>(static_cast<const char*>(ddesc_[slot].ptr) + db), R, st_));
  ++launches_;
  HZ_CUDA(cudaEventRecord(done_, st_));
  for (const Req* r : batch) HZ_CUDA(cudaStreamWaitEvent(r->st, done_, 0));
  return HZ_OK;
}

}  // namespace hz
