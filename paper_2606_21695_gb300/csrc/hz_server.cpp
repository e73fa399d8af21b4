// Request server: continuous batching of Helmholtz solves on one device.
//
// submit() snapshots the problem's fields into host memory and queues the
// request; nothing of a queued request lives on the device.  A pool of worker
// threads admits queued requests whenever a request's estimated device
// footprint fits in the HBM budget (first fit in arrival order; a request
// passed over too often blocks the ones behind it until it fits, so large
// requests are not starved), and only then copies its fields to the device.
// Each admitted solve runs on its own CUDA stream, and with opts.pack the
// sweeps of all admitted solves go out together, one packed launch per outer
// step (hz_pack.cpp), so a request that arrives while others run is admitted
// as soon as a worker and memory free up and joins the next packed launch.
// Latency is measured from submit() to the completed device-to-host copy of u.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hz_admission.h"
#include "hz_internal.h"
#include "hz_pack.h"
#include "hz_problem.h"

using namespace hz;

namespace {

using clk = std::chrono::steady_clock;

// Device buffers of a problem that carry its fields (the rest is solver
// workspace, sized by the solve itself).
using BufMember = DevBuf hz_problem_s::*;
constexpr BufMember kFieldBufs[] = {&hz_problem_s::c,      &hz_problem_s::f,      &hz_problem_s::gb,
                                    &hz_problem_s::Wxg,    &hz_problem_s::Wyg,    &hz_problem_s::wxs,
                                    &hz_problem_s::wys,    &hz_problem_s::mgeo64, &hz_problem_s::mgeo32,
                                    &hz_problem_s::mWs,    &hz_problem_s::mEs,    &hz_problem_s::mshare,
                                    &hz_problem_s::mgeog,  &hz_problem_s::mWg,    &hz_problem_s::mHw,
                                    &hz_problem_s::mbw};
constexpr int kNumFieldBufs = (int)(sizeof(kFieldBufs) / sizeof(kFieldBufs[0]));
// A request passed over this many times by first-fit admission blocks the
// queue behind it until it fits.
constexpr int kMaxPassOver = 64;

struct Request {
  uint64_t ticket = 0;
  std::unique_ptr<hz_problem_s> pr;  // scalars from submit; device buffers only once admitted
  std::vector<std::vector<unsigned char>> host;  // field snapshot, one per kFieldBufs entry
  size_t flux_bytes = 0;             // mapped meshes: residual flux scratch to allocate
  int passed_over = 0;
  hz_solve_opts opts{};
  uint64_t bytes = 0;
  clk::time_point t_submit;
  // result
  bool done = false;
  hz_status status = HZ_OK;
  std::string error;
  hz_solve_report report{};
  std::vector<double> u;
};

uint64_t estimate_bytes(const Geom& g, const hz_solve_opts& o, bool mapped = false) {
  const uint64_t n = (uint64_t)g.n, ns = (uint64_t)g.L * g.sub_nodes(), nl = (uint64_t)g.lam_complex();
  uint64_t b = 0;
  if (mapped) {  // metric per element node (subdomain FP64 + FP32, global FP64), flux scratch, weights
    const uint64_t en = (uint64_t)g.nx * g.ny * (g.P + 1) * (g.P + 1);
    b += en * (24 + 12 + 24 + 32) + ns * 16 + nl * 8 + n * 16;
  }
  if (o.wh_warm) b += ns * 16;  // warm-start subdomain solutions
  if (o.refine == HZ_REFINE_FGMRES)  // global Krylov and preconditioned vectors of a cycle
    b += n * 16 * (uint64_t)(2 * std::max(1, o.refine_restart) + 1);
  b += n * 8 + n * 16 + (uint64_t)(2 * g.NXg + 2 * g.NYg) * 16;  // c, f, g
  b += 3 * n * 16;                                                 // b, r, u
  b += ns * 16 + ns * 24;                                          // u_sub, alpha/beta (64 + 32 bit)
  b += nl * 8 + nl * 16 * (uint64_t)(o.gmres_restart + 4);         // kedge, lambda vectors
  b += (uint64_t)1 << 20;                                          // tables, partial sums
  return b;
}

// Host snapshot of a problem: its scalars and a copy of every field buffer.
// Queued requests hold no device memory.
hz_status snapshot_problem(const hz_problem_s& src, Request* req) {
  auto pr = std::make_unique<hz_problem_s>();
  pr->g = src.g;
  pr->device = src.device;
  pr->omega = src.omega;
  pr->cmax = src.cmax;
  pr->robin_eta = src.robin_eta;
  pr->robin_zeta = src.robin_zeta;
  pr->has_c = src.has_c;
  pr->has_omega = src.has_omega;
  pr->mapped = src.mapped;
  pr->mapped_mu = src.mapped_mu;
  pr->mapped_D = src.mapped_D;
  HZ_CUDA(cudaSetDevice(src.device));
  req->host.assign(kNumFieldBufs, {});
  for (int k = 0; k < kNumFieldBufs; ++k) {
    const DevBuf& b = src.*kFieldBufs[k];
    if (!b.ptr) continue;
    try {
      req->host[k].resize(b.bytes);
    } catch (...) {
      return fail(HZ_ERR_OOM, "host snapshot of the problem failed");
    }
    HZ_CUDA(cudaMemcpy(req->host[k].data(), b.ptr, b.bytes, cudaMemcpyDeviceToHost));
  }
  req->flux_bytes = src.mapped ? src.mflux.bytes : 0;
  req->pr = std::move(pr);
  return HZ_OK;
}

// Gives an admitted request a stream and copies its fields to the device on
// it (the solve that follows on the same stream is ordered after the copies;
// the stream is synchronised before the host snapshot is dropped).
hz_status materialize(Request* req) {
  hz_problem_s& pr = *req->pr;
  HZ_CUDA(cudaSetDevice(pr.device));
  HZ_CUDA(cudaStreamCreateWithFlags(&pr.stream, cudaStreamNonBlocking));
  for (int k = 0; k < kNumFieldBufs; ++k) {
    std::vector<unsigned char>& h = req->host[k];
    if (h.empty()) continue;
    DevBuf& d = pr.*kFieldBufs[k];
    HZ_TRY(d.ensure(h.size()));
    HZ_CUDA(cudaMemcpyAsync(d.ptr, h.data(), h.size(), cudaMemcpyHostToDevice, pr.stream));
  }
  HZ_CUDA(cudaStreamSynchronize(pr.stream));
  for (auto& h : req->host) std::vector<unsigned char>().swap(h);
  if (req->flux_bytes) HZ_TRY(pr.mflux.ensure(req->flux_bytes));
  return HZ_OK;
}

}  // namespace

struct hz_server_s {
  int device = 0;
  uint64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_ticket = 1;
  uint64_t in_use = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies_ms;
  uint64_t completed = 0;
  std::unique_ptr<Packer> packer;  // sweeps of concurrently served solves, one launch per step
  clk::time_point t_start = clk::now();

  // First queued request that fits in the budget (removed from the queue), or
  // null (hz_admission.h).
  Request* pick() { return first_fit(queue, in_use, budget, kMaxPassOver); }

  void worker_loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      Request* job = nullptr;
      cv_work.wait(lk, [&] {
        if (stopping) return true;
        job = pick();
        return job != nullptr;
      });
      if (stopping) return;
      in_use += job->bytes;
      lk.unlock();
      // copy the fields to the device now that the budget holds them, then
      // run the solve on the request's own stream
      hz_problem_s& pr = *job->pr;
      const size_t nb = (size_t)pr.g.n * 2 * sizeof(double);
      hz_status s = materialize(job);
      if (s == HZ_OK) s = pr.uvec.ensure(nb);
      hz_solve_report rep{};
      const bool packed = job->opts.pack && packer && Packer::packable(pr, job->opts);
      if (packed) {
        pr.packer = packer.get();
        packer->join();
      }
      if (s == HZ_OK) s = hz::solve(pr, job->opts, pr.uvec.as<double>(), &rep, pr.stream);
      if (packed) {
        packer->leave();
        pr.packer = nullptr;
      }
      std::vector<double> u;
      if (s == HZ_OK || s == HZ_ERR_NOT_CONVERGED) {
        u.resize((size_t)pr.g.n * 2);
        if (cudaMemcpyAsync(u.data(), pr.uvec.ptr, nb, cudaMemcpyDeviceToHost, pr.stream) != cudaSuccess ||
            cudaStreamSynchronize(pr.stream) != cudaSuccess) {
          (void)cudaGetLastError();
          s = fail(HZ_ERR_CUDA, "copy of the solution failed");
        }
      }
      char msg[512] = {0};
      if (s != HZ_OK) hz_last_error(msg, sizeof msg);
      const double ms = std::chrono::duration<double, std::milli>(clk::now() - job->t_submit).count();
      // release device memory before admitting the next request
      const uint64_t freed = job->bytes;
      for (cudaEvent_t e : pr.events) cudaEventDestroy(e);
      pr.events.clear();
      for (cudaEvent_t e : pr.gm_events) cudaEventDestroy(e);
      pr.gm_events.clear();
      if (pr.pack_ready) cudaEventDestroy(pr.pack_ready);
      pr.pack_ready = nullptr;
      release_step_graphs(pr);
      if (pr.stream) cudaStreamDestroy(pr.stream);
      pr.stream = nullptr;
      job->pr.reset();
      lk.lock();
      job->status = s;
      job->error = msg;
      job->report = rep;
      job->u.swap(u);
      job->done = true;
      in_use -= freed;
      latencies_ms.push_back(ms);
      completed++;
      cv_done.notify_all();
      cv_work.notify_all();
    }
  }
};

extern "C" {

hz_status hz_server_create(int32_t device, uint64_t hbm_budget_bytes, hz_server* out) {
  if (!out) return fail(HZ_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  int ndev = 0;
  HZ_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(HZ_ERR_INVALID_ARG, "no such CUDA device");
  if (hbm_budget_bytes == 0) return fail(HZ_ERR_INVALID_ARG, "HBM budget must be > 0");
  HZ_CUDA(cudaSetDevice(device));
  std::unique_ptr<hz_server_s> s;
  try {
    s = std::make_unique<hz_server_s>();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->packer = std::make_unique<Packer>(device);
  } catch (...) {
    return fail(HZ_ERR_INTERNAL, "could not create the server");
  }
  const char* env = std::getenv("HZ_SERVER_WORKERS");
  int nw = env ? std::atoi(env) : 8;
  nw = std::max(1, std::min(nw, 32));
  try {
    for (int k = 0; k < nw; ++k) s->workers.emplace_back([p = s.get()] { p->worker_loop(); });
  } catch (...) {  // stop the workers that did start before the server goes away
    hz_server_destroy(s.release());
    return fail(HZ_ERR_INTERNAL, "could not start the server's worker threads");
  }
  *out = s.release();
  return HZ_OK;
}

hz_status hz_server_submit(hz_server srv, hz_problem pr, const hz_solve_opts* opts, uint64_t* ticket) {
  if (!srv || !pr || !ticket) return fail(HZ_ERR_INVALID_ARG, "null argument");
  HZ_TRY(check_ready(*pr));
  auto req = std::make_unique<Request>();
  if (opts) req->opts = *opts;
  else hz_default_opts(&req->opts);
  req->bytes = estimate_bytes(pr->g, req->opts, pr->mapped);
  if (req->bytes > srv->budget) return fail(HZ_ERR_BUSY, "request larger than the server's HBM budget");
  HZ_TRY(snapshot_problem(*pr, req.get()));
  req->t_submit = clk::now();
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stopping) return fail(HZ_ERR_BUSY, "server is shutting down");
  req->ticket = srv->next_ticket++;
  *ticket = req->ticket;
  srv->queue.push_back(req.get());
  srv->reqs[req->ticket] = std::move(req);
  srv->cv_work.notify_one();
  return HZ_OK;
}

hz_status hz_server_poll(hz_server srv, uint64_t ticket, int32_t timeout_ms, double* u_out, hz_solve_report* report,
                         int32_t* done) {
  if (!srv || !done) return fail(HZ_ERR_INVALID_ARG, "null argument");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return fail(HZ_ERR_NOT_FOUND, "unknown ticket");
  Request* r = it->second.get();
  auto ready = [&] { return r->done; };
  if (!r->done) {
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else if (timeout_ms > 0) srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  if (!r->done) {
    *done = 0;
    return timeout_ms > 0 ? fail(HZ_ERR_TIMEOUT, "request not finished within the timeout") : HZ_OK;
  }
  *done = 1;
  if (u_out && !r->u.empty()) std::memcpy(u_out, r->u.data(), r->u.size() * sizeof(double));
  if (report) *report = r->report;
  const hz_status s = r->status;
  if (s != HZ_OK) set_error(r->error);
  srv->reqs.erase(it);
  return s;
}

hz_status hz_server_stats(hz_server srv, double* p50_ms, double* p99_ms, double* solves_per_s, uint64_t* hbm_in_use) {
  if (!srv) return fail(HZ_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(srv->mu);
  std::vector<double> v = srv->latencies_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5));
    return v[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  const double el = std::chrono::duration<double>(clk::now() - srv->t_start).count();
  if (solves_per_s) *solves_per_s = el > 0 ? srv->completed / el : 0.0;
  if (hbm_in_use) *hbm_in_use = srv->in_use;
  return HZ_OK;
}

void hz_server_destroy(hz_server srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  delete srv;
}

}  // extern "C"
