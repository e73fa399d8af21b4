// Batched solves: many independent problems on one device at once.
//
// Each problem keeps its own device state and stream; a pool of host
// threads advances the solves concurrently.  With opts.pack the sweeps of the
// running solves go out together: one packed launch per outer step covers
// every subdomain of every member (different sizes, degrees and frequencies;
// hz_pack.cpp), otherwise each solve launches its own sweeps and they overlap
// on the GPU.  Either way small problems fill the SMs that one of them alone
// would leave idle.  Problems start in decreasing order of estimated cost
// (longest processing time first: subdomain nodes x (N_t - 1) x WaveHoltz
// iterations), and the sweep kernel of every distinct subdomain shape is
// autotuned once, before the concurrent phase, so the timings are not
// disturbed by the other solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "hz_internal.h"
#include "hz_pack.h"
#include "hz_problem.h"

using namespace hz;

extern "C" hz_status hz_solve_batch(const hz_problem* problems, int32_t count, const hz_solve_opts* opts,
                                     int32_t max_concurrent, double* const* u_out, hz_solve_report* reports,
                                     hz_status* statuses) {
  if (!problems || count < 0 || !statuses) return fail(HZ_ERR_INVALID_ARG, "null argument or negative count");
  if (count == 0) return HZ_OK;
  hz_solve_opts o;
  if (opts) o = effective_opts(*opts);
  else hz_default_opts(&o);
  for (int k = 0; k < count; ++k) {
    if (!problems[k]) return fail(HZ_ERR_INVALID_ARG, "null problem in batch");
    HZ_TRY(check_ready(*problems[k]));
    for (int q = 0; q < k; ++q)
      if (problems[q] == problems[k]) return fail(HZ_ERR_INVALID_ARG, "a problem appears twice in the batch");
  }
  // estimated cost and LPT order
  std::vector<std::pair<double, int>> order;
  std::vector<int> nts(count);
  for (int k = 0; k < count; ++k) {
    Problem& pr = *problems[k];
    nts[k] = o.nt_override > 0 ? o.nt_override : choose_nt(pr, o.cfl);
    const double cost = (double)pr.g.L * pr.g.sub_nodes() * (nts[k] - 1) * o.wh_iters;
    order.emplace_back(-cost, k);
  }
  std::sort(order.begin(), order.end());
  // autotune each distinct shape once, sequentially
  if (o.autotune && sweep_variant() == kVariantAuto) {
    std::vector<std::string> seen;
    for (auto& [c, k] : order) {
      Problem& pr = *problems[k];
      const std::string key = tune_key(pr.g, o.precision);
      if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
      seen.push_back(key);
      HZ_CUDA(cudaSetDevice(pr.device));
      HZ_TRY(autotune(pr, o.precision, nts[k], o.wh_iters, pr.stream));
    }
  }
  int nw = max_concurrent > 0 ? max_concurrent : 64;
  nw = std::max(1, std::min(nw, count));
  // one packer per device in use
  std::map<int, std::unique_ptr<Packer>> packers;
  if (o.pack) {
    for (int k = 0; k < count; ++k) {
      Problem& pr = *problems[k];
      if (!Packer::packable(pr, o) || packers.count(pr.device)) continue;
      HZ_CUDA(cudaSetDevice(pr.device));
      packers[pr.device] = std::make_unique<Packer>(pr.device);
    }
  }
  std::atomic<int> next{0};
  std::vector<std::string> errors(count);
  auto worker = [&]() {
    while (true) {
      const int idx = next.fetch_add(1);
      if (idx >= count) return;
      const int k = order[idx].second;
      Problem& pr = *problems[k];
      hz_status s = HZ_OK;
      if (cudaSetDevice(pr.device) != cudaSuccess) s = fail(HZ_ERR_CUDA, "cudaSetDevice failed");
      const size_t nb = (size_t)pr.g.n * 2 * sizeof(double);
      if (s == HZ_OK) s = pr.uvec.ensure(nb);
      hz_solve_report rep{};
      Packer* pk = nullptr;
      if (o.pack && Packer::packable(pr, o)) {
        pk = packers.at(pr.device).get();
        pr.packer = pk;
        pk->join();
      }
      if (s == HZ_OK) s = solve(pr, o, pr.uvec.as<double>(), &rep, pr.stream);
      if (pk) {
        pk->leave();
        pr.packer = nullptr;
      }
      if ((s == HZ_OK || s == HZ_ERR_NOT_CONVERGED) && u_out && u_out[k]) {
        if (cudaMemcpyAsync(u_out[k], pr.uvec.ptr, nb, cudaMemcpyDeviceToHost, pr.stream) != cudaSuccess ||
            cudaStreamSynchronize(pr.stream) != cudaSuccess) {
          (void)cudaGetLastError();
          s = fail(HZ_ERR_CUDA, "copy of the solution failed");
        }
      }
      if (s != HZ_OK) {
        char msg[512] = {0};
        hz_last_error(msg, sizeof msg);
        errors[k] = msg;
      }
      statuses[k] = s;
      if (reports) reports[k] = rep;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < nw; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  hz_status worst = HZ_OK;
  for (int k = 0; k < count; ++k) {
    if (statuses[k] != HZ_OK && statuses[k] != HZ_ERR_NOT_CONVERGED) {
      worst = statuses[k];
      set_error("problem " + std::to_string(k) + ": " + errors[k]);
    } else if (statuses[k] == HZ_ERR_NOT_CONVERGED && worst == HZ_OK) {
      worst = HZ_ERR_NOT_CONVERGED;
    }
  }
  return worst;
}
