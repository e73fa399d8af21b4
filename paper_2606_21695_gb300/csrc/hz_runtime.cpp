// Host runtime behind the C ABI: problem state, coefficient preparation,
// the sweep kernel choice and its autotuner, the outer iteration on the
// transmission data (GMRES / plain / real GMRES, Sec. 3), the FP64
// refinement on the global residual (defect correction or flexible GMRES,
// Sec. 7), and the extern "C" entry points declared in include/hz.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hz_internal.h"
#include "hz_pack.h"
#include "hz_problem.h"

namespace hz {

// ------------------------------------------------------------- errors ----
namespace {
thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
void set_error(const std::string& msg) { g_last_error = msg; }
hz_status fail(hz_status s, const std::string& msg) {
  set_error(msg);
  return s;
}
hz_status cuda_fail(cudaError_t e, const char* what) {
  return fail(HZ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

hz_status DevBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && ptr) return HZ_OK;
  release();
  if (nbytes == 0) nbytes = 16;
  cudaError_t e = cudaMalloc(&ptr, nbytes);
  if (e != cudaSuccess) {
    ptr = nullptr;
    bytes = 0;
    (void)cudaGetLastError();
    return fail(HZ_ERR_OOM, std::string("device allocation of ") + std::to_string(nbytes) + " bytes failed: " +
                                cudaGetErrorString(e));
  }
  bytes = nbytes;
  return HZ_OK;
}
void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

HostBuf::~HostBuf() {
  if (ptr) cudaFreeHost(ptr);
}
hz_status HostBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && ptr) return HZ_OK;
  if (ptr) cudaFreeHost(ptr);
  ptr = nullptr;
  bytes = 0;
  if (cudaHostAlloc(&ptr, nbytes, cudaHostAllocDefault) != cudaSuccess) {
    ptr = nullptr;
    (void)cudaGetLastError();
    return fail(HZ_ERR_OOM, "pinned host allocation failed");
  }
  bytes = nbytes;
  return HZ_OK;
}

// ---------------------------------------------------------- problem ops ----
int choose_nt(const Problem& pr, double cfl) {
  const Geom& g = pr.g;
  // Cartesian: lambda_max(M^-1 A) of the subdomain from its 1D factors;
  // mapped: the element bound (power iteration per element, 1% margin)
  const double lam = pr.mapped ? pr.cmax * pr.cmax * pr.mapped_mu * 1.01
                               : pr.cmax * pr.cmax * (max_eig_1d(g, g.snx, g.hx) + max_eig_1d(g, g.sny, g.hy));
  const double dt_max = cfl * 2.0 / std::sqrt(lam);
  const double T = 2.0 * M_PI / pr.omega;
  const double q = std::ceil(T / dt_max);
  return std::max(3, (int)q);
}

static GlobalArgs global_args(const Problem& pr) {
  const Geom& g = pr.g;
  GlobalArgs a{};
  a.NXg = g.NXg;
  a.NYg = g.NYg;
  a.nx = g.nx;
  a.ny = g.ny;
  a.P = g.P;
  a.omega = pr.omega;
  a.kxs = 2.0 / g.hx;
  a.kys = 2.0 / g.hy;
  a.hx2 = g.hx / 2.0;
  a.hy2 = g.hy / 2.0;
  for (size_t k = 0; k < g.Kref.size(); ++k) a.Kref[k] = g.Kref[k];
  for (int k = 0; k <= g.P; ++k) a.w[k] = g.w[k];
  // assembled rows: class c < P is an element's node c (c = 0: also node P of
  // the element to the left); class P the mesh's first node (own element
  // only), class P+1 its last node (left element only)
  const int P = g.P;
  for (int c = 0; c < P + 2; ++c)
    for (int tt = -P; tt <= P; ++tt) {
      const int ax = c < P ? c : (c == P ? 0 : P);
      const bool own = c <= P, left = (c == 0 || c == P + 1);
      double v = 0.0;
      const int bb = ax + tt;
      if (own && bb >= 0 && bb <= P) v += g.Kref[(size_t)ax * (P + 1) + bb];
      if (left && tt <= 0) v += g.Kref[(size_t)P * (P + 1) + (tt + P)];
      a.Kx[c][tt + P] = v * a.kxs;
      a.Ky[c][tt + P] = v * a.kys;
    }
  a.c = pr.c.as<double>();
  a.Wxg = pr.Wxg.as<double>();
  a.Wyg = pr.Wyg.as<double>();
  return a;
}

bool is_default_stream(cudaStream_t s) { return s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread; }

void release_step_graphs(Problem& pr) {
  for (cudaGraphExec_t g : pr.step_graphs)
    if (g) cudaGraphExecDestroy(g);
  pr.step_graphs.clear();
  pr.step_graph_kernels.clear();
  pr.step_graph_key.clear();
}

hz_status check_ready(const Problem& pr) {
  if (!pr.has_c) return fail(HZ_ERR_INVALID_ARG, "wave speed not set");
  if (!pr.has_omega) return fail(HZ_ERR_INVALID_ARG, "omega not set");
  return HZ_OK;
}

hz_status prepare(Problem& pr, int nt, cudaStream_t st) {
  HZ_TRY(check_ready(pr));
  if (nt < 3) return fail(HZ_ERR_INVALID_ARG, "N_t must be >= 3");
  if (pr.prepared_nt == nt && pr.prepared_version == pr.version) return HZ_OK;
  const Geom& g = pr.g;
  const int64_t nsub = (int64_t)g.L * g.sub_nodes();
  HZ_TRY(pr.beta64.ensure(nsub * sizeof(double)));
  HZ_TRY(pr.alpha64.ensure(nsub * sizeof(double)));
  HZ_TRY(pr.beta32.ensure(nsub * sizeof(float)));
  HZ_TRY(pr.alpha32.ensure(nsub * sizeof(float)));
  HZ_TRY(pr.kedge.ensure((size_t)g.lam_complex() * sizeof(double)));
  const double w = pr.omega;
  const double dt = (2.0 * M_PI / w) / nt;
  PrepArgs a{};
  a.nlx = g.nlx;
  a.nly = g.nly;
  a.NE = g.NE;
  a.Sx = g.Sx;
  a.Sy = g.Sy;
  a.NXg = g.NXg;
  a.snxP = g.snx * g.P;
  a.snyP = g.sny * g.P;
  a.theta = std::tan(w * dt / 2.0) / w;
  a.sigma = std::sin(w * dt / 2.0) / (w / 2.0);
  a.omega = w;
  a.zeta = pr.robin_zeta;
  a.c = pr.c.as<double>();
  a.wxs = pr.wxs.as<double>();
  a.wys = pr.wys.as<double>();
  a.Wsub = pr.mapped ? pr.mWs.as<double>() : nullptr;
  a.Esub = pr.mapped ? pr.mEs.as<double>() : nullptr;
  a.beta64 = pr.beta64.as<double>();
  a.alpha64 = pr.alpha64.as<double>();
  a.beta32 = pr.beta32.as<float>();
  a.alpha32 = pr.alpha32.as<float>();
  a.kedge = pr.kedge.as<double>();
  HZ_TRY(launch_prepare(a, g.L, st));
  // filter / forcing tables: nu = 0..Nt: cos, sin of 2 pi nu/Nt, kappa_nu, kappa_{nu+1/2}/omega
  const double c0 = -0.25 + 0.25 * std::tan(M_PI / nt) * std::tan(M_PI / nt);
  std::vector<double> t64(4 * (size_t)(nt + 1));
  std::vector<float> t32(4 * (size_t)(nt + 1));
  for (int nu = 0; nu <= nt; ++nu) {
    const double th = 2.0 * M_PI * nu / nt;
    t64[4 * nu + 0] = std::cos(th);
    t64[4 * nu + 1] = std::sin(th);
    t64[4 * nu + 2] = std::cos(th) + c0;
    t64[4 * nu + 3] = (std::cos(2.0 * M_PI * (nu + 0.5) / nt) + c0) / w;
    for (int k = 0; k < 4; ++k) t32[4 * nu + k] = (float)t64[4 * nu + k];
  }
  HZ_TRY(pr.tab64.ensure(t64.size() * sizeof(double)));
  HZ_TRY(pr.tab32.ensure(t32.size() * sizeof(float)));
  HZ_CUDA(cudaMemcpyAsync(pr.tab64.ptr, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  HZ_CUDA(cudaMemcpyAsync(pr.tab32.ptr, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  HZ_CUDA(cudaStreamSynchronize(st));  // host tables go out of scope
  pr.prepared_nt = nt;
  pr.prepared_version = pr.version;
  pr.sigma = a.sigma;
  return HZ_OK;
}

hz_status ensure_flags(Problem& pr) {
  if (!pr.flags.ptr) {
    HZ_TRY(pr.flags.ensure(64));
    HZ_CUDA(cudaMemset(pr.flags.ptr, 0, 64));
  }
  return HZ_OK;
}

// Sweep kernel selection: HZ_SWEEP_VARIANT=block|warp|cluster forces one (tests);
// default: the warp-per-subdomain kernel when compiled for the shape, else
// the block kernel.
int sweep_variant() {
  const char* v = std::getenv("HZ_SWEEP_VARIANT");
  if (!v) return kVariantAuto;
  if (std::strcmp(v, "block") == 0) return kVariantBlock;
  if (std::strcmp(v, "warp") == 0) return kVariantWarp;
  if (std::strcmp(v, "cluster") == 0) return kVariantCluster;
  if (std::strcmp(v, "cband") == 0) return kVariantClusterBand;
  return kVariantAuto;
}

// Row weights of a subdomain and the y scale for the register-resident kernels.
void warp_rows(const Geom& g, WarpSweepArgs* w) {
  const int P = g.P;
  w->sy = (float)(4.0 / (g.hy * g.hy));
  for (int j = 0; j < kWarpMaxRows; ++j) {
    const int ay = j % P, ey = j / P;
    const bool own = ey < g.sny, below = ay == 0 && ey >= 1;
    w->wyr[j] = (float)(g.hy / 2.0 * ((own ? g.w[ay] : 0.0) + (below ? g.w[P] : 0.0)));
  }
}

// ---- sweep kernel choices and the autotuner's cache
namespace {
std::mutex g_tune_mu;
std::map<std::string, Choice> g_tuned;
}  // namespace

std::string tune_key(const Geom& g, int precision) {
  int lb = 0;
  while ((1 << (lb + 1)) <= g.L) ++lb;  // occupancy depends on the number of subdomains
  return std::to_string(g.P) + "/" + std::to_string(g.nlx) + "x" + std::to_string(g.nly) + "/L2^" +
         std::to_string(lb) + "/" + std::to_string(precision);
}

bool lookup_choice(const std::string& key, Choice* out) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(key);
  if (it == g_tuned.end()) return false;
  *out = it->second;
  return true;
}

void store_choice(const std::string& key, Choice c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = c;
}

hz_status launch_choice(Problem& pr, const SweepArgs& a0, Choice c, bool fp32, cudaStream_t st) {
  const Geom& g = pr.g;
  const int count = sweep_count(a0, g.L);
  hz_status s = HZ_ERR_UNSUPPORTED;
  if (c.variant == kVariantWarp) {
    if (!fp32) return HZ_ERR_UNSUPPORTED;
    WarpSweepArgs w{};
    w.base = a0;
    w.L = count;
    warp_rows(g, &w);
    s = launch_sweep_warp(g.P, g.sny, c.ty > 0 ? c.ty : 1, w, st);
  } else if (c.variant == kVariantClusterBand) {
    if (!fp32) return HZ_ERR_UNSUPPORTED;
    SweepArgs a = a0;
    a.ty_force = c.ty;  // 8: 8 rows per warp band, else 16
    s = launch_sweep_cband(g.P, a, count, st);
  } else if (c.variant == kVariantCluster) {
    if (a0.round_mode != 0) return HZ_ERR_UNSUPPORTED;  // 16-bit trials run on the block kernel
    SweepArgs a = a0;
    a.ty_force = c.ty;  // 4: 4P rows per thread, else 2P
    s = fp32 ? launch_sweep_cluster(g.P, a, count, st) : launch_sweep_cluster_f64(g.P, a, count, st);
  } else {
    SweepArgs a = a0;
    a.ty_force = c.ty;
    s = launch_sweep(fp32, g.P, a, count, st);
  }
  if (s == HZ_OK) {
    pr.last_variant = c.variant;
    pr.last_shape = c.variant == kVariantWarp ? (c.ty > 0 ? c.ty : 1) : c.ty;
  }
  return s;
}

SweepArgs make_sweep_args(Problem& pr, bool fp32, int nt, int m_wh, double wh_tol, const double* lam_in,
                          double* lam_out, const double* rhs, double* u_sub) {
  const Geom& g = pr.g;
  SweepArgs a{};
  a.nlx = g.nlx;
  a.nly = g.nly;
  a.NE = g.NE;
  a.Sx = g.Sx;
  a.Sy = g.Sy;
  a.sxe = g.snx;
  a.sye = g.sny;
  a.NXg = g.NXg;
  a.snxP = g.snx * g.P;
  a.snyP = g.sny * g.P;
  a.Nt = nt;
  a.m_wh = m_wh;
  a.wh_tol = wh_tol;
  a.sigma = pr.sigma;
  a.omega = pr.omega;
  a.cpi = std::cos(M_PI / nt);
  a.spi = std::sin(M_PI / nt);
  a.two_over_nt = 2.0 / nt;
  a.kxs = 2.0 / g.hx;
  a.kys = 2.0 / g.hy;
  a.hx2 = g.hx / 2.0;
  a.hy2 = g.hy / 2.0;
  a.eta = pr.robin_eta;
  a.zeta = pr.robin_zeta;
  for (size_t k = 0; k < g.Kref.size(); ++k) {
    a.Kref[k] = g.Kref[k];
    a.Kref32[k] = (float)g.Kref[k];
  }
  for (int k = 0; k <= g.P; ++k) a.w[k] = g.w[k];
  a.beta = fp32 ? pr.beta32.ptr : pr.beta64.ptr;
  a.alpha = fp32 ? pr.alpha32.ptr : pr.alpha64.ptr;
  a.tab = fp32 ? pr.tab32.ptr : pr.tab64.ptr;
  a.kedge = pr.kedge.as<double>();
  a.wxs = pr.wxs.as<double>();
  a.wys = pr.wys.as<double>();
  a.rhs = rhs;
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.u_sub = u_sub;
  int* fl = pr.flags.as<int>();
  a.flags = fl;
  a.wh_iter_max = fl + 1;
  a.wh_iter_sum = reinterpret_cast<unsigned long long*>(fl + 2);
  return a;
}

namespace {
std::mutex g_tune_run_mu;
}

// Autotuner: times every sweep kernel variant that supports the shape (warp
// per subdomain; one block per subdomain with P or 2P rows per thread; a
// cluster of blocks) on this problem and caches the fastest per shape key.
hz_status autotune(Problem& pr, int precision, int nt, int m_wh, cudaStream_t st) {
  const std::string key = tune_key(pr.g, precision);
  Choice c{};
  if (lookup_choice(key, &c)) return HZ_OK;
  std::lock_guard<std::mutex> lk(g_tune_run_mu);
  if (lookup_choice(key, &c)) return HZ_OK;
  HZ_TRY(prepare(pr, nt, st));
  HZ_TRY(ensure_flags(pr));
  const size_t vb = (size_t)pr.g.lam_complex() * 2 * sizeof(double);
  HZ_TRY(pr.xv.ensure(vb));
  HZ_TRY(pr.tv.ensure(vb));
  HZ_CUDA(cudaMemsetAsync(pr.xv.ptr, 0, vb, st));
  const bool fp32 = precision == HZ_FP32_REFINE;
  const SweepArgs a = make_sweep_args(pr, fp32, nt, m_wh, 0.0, pr.xv.as<double>(), pr.tv.as<double>(), nullptr, nullptr);
  std::vector<Choice> cands;
  if (fp32)
    cands = {{kVariantWarp, 1}, {kVariantWarp, 2}, {kVariantWarp, 4}, {kVariantBlock, 1}, {kVariantBlock, 2},
             {kVariantCluster, 0}, {kVariantCluster, 4}, {kVariantClusterBand, 0}, {kVariantClusterBand, 8}};
  else cands = {{kVariantBlock, 1}, {kVariantBlock, 2}, {kVariantCluster, 0}, {kVariantCluster, 4}};
  cudaEvent_t e0, e1;
  HZ_CUDA(cudaEventCreate(&e0));
  HZ_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  Choice bc{kVariantBlock, 0};
  for (const Choice& cand : cands) {
    hz_status s = launch_choice(pr, a, cand, fp32, st);  // warm-up, also the support check
    if (s == HZ_ERR_UNSUPPORTED) continue;
    if (s != HZ_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return s;
    }
    cudaEventRecord(e0, st);
    for (int k = 0; k < 2; ++k) launch_choice(pr, a, cand, fp32, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (std::getenv("HZ_TUNE_LOG"))
      std::fprintf(stderr, "hz autotune %s: candidate %d/%d %.4f ms per sweep\n", key.c_str(), cand.variant, cand.ty,
                   ms / 2);
    if (ms < best) {
      best = ms;
      bc = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HZ_CUDA(cudaGetLastError());
  store_choice(key, bc);
  if (std::getenv("HZ_TUNE_LOG"))
    std::fprintf(stderr, "hz autotune %s: variant %d/%d, %.4f ms per sweep\n", key.c_str(), bc.variant, bc.ty, best / 2);
  return HZ_OK;
}

hz_status sweep(Problem& pr, int precision, int nt, int m_wh, double wh_tol, const double* lam_in, double* lam_out,
                const double* rhs, double* u_sub, cudaStream_t st, const double* u0, const int* rect) {
  HZ_TRY(prepare(pr, nt, st));
  HZ_TRY(ensure_flags(pr));
  const Geom& g = pr.g;
  if (m_wh < 0) return fail(HZ_ERR_INVALID_ARG, "wh_iters must be >= 0");
  if (precision < HZ_FP64 || precision > HZ_BF16_TRIAL) return fail(HZ_ERR_INVALID_ARG, "unknown precision");
  const bool trial = precision == HZ_FP16_TRIAL || precision == HZ_BF16_TRIAL;
  const bool fp32 = precision != HZ_FP64;
  SweepArgs a = make_sweep_args(pr, fp32, nt, m_wh, wh_tol, lam_in, lam_out, rhs, u_sub);
  if (rect) {  // rank-local sweep of a rectangle of subdomains
    a.rect_x0 = rect[0];
    a.rect_y0 = rect[1];
    a.rect_w = rect[2];
    a.rect_h = rect[3];
  }
  const int count = sweep_count(a, g.L);
  if (trial) a.round_mode = precision == HZ_FP16_TRIAL ? 1 : 2;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (pr.time_sweeps) {
    if (pr.ev_used + 2 > pr.events.size()) {
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t e;
        HZ_CUDA(cudaEventCreate(&e));
        pr.events.push_back(e);
      }
    }
    e0 = pr.events[pr.ev_used];
    e1 = pr.events[pr.ev_used + 1];
    pr.ev_used += 2;
    HZ_CUDA(cudaEventRecord(e0, st));
  }
  // general convex quadrilaterals: the element-form kernel (one variant)
  if (pr.mapped) {
    if (trial) return fail(HZ_ERR_UNSUPPORTED, "16-bit trials are not built for mapped meshes");
    MappedSweepArgs ma{};
    ma.base = a;
    ma.base.u0 = u0;
    ma.geo = fp32 ? pr.mgeo32.ptr : pr.mgeo64.ptr;
    ma.wedge = pr.mEs.as<double>();
    ma.share = pr.mshare.as<double>();
    ma.snx = g.snx;
    ma.sny = g.sny;
    for (size_t k = 0; k < pr.mapped_D.size(); ++k) ma.D[k] = pr.mapped_D[k];
    HZ_TRY(launch_sweep_mapped(fp32, g.P, ma, count, st));
    pr.last_variant = kVariantMapped;
    pr.last_shape = 0;
    if (e1) HZ_CUDA(cudaEventRecord(e1, st));
    pr.sweeps_launched++;
    return HZ_OK;
  }
  // A solve running as a member of a packer hands its sweep over: one packed
  // launch per outer step covers the subdomains of every member.
  if (pr.packer && precision == HZ_FP32_REFINE && !(wh_tol > 0.0) && !u0 && !rect) {
    const int shape = packed_shape_id(g.P, g.sny, g.nlx);
    if (shape >= 0) {
      WarpSweepArgs w{};
      w.base = a;
      w.L = g.L;
      warp_rows(g, &w);
      HZ_TRY(pr.packer->submit(pr, w, shape, st));
      pr.last_variant = kVariantPacked;
      pr.last_shape = 1;
      if (e1) HZ_CUDA(cudaEventRecord(e1, st));
      pr.sweeps_launched++;
      return HZ_OK;
    }
  }
  // Kernel choice: HZ_SWEEP_VARIANT forces a variant; otherwise the tuned
  // choice for this shape (if autotuning ran) or the size heuristic:
  // FP32 -> warp-per-subdomain kernel when compiled for the shape, else one
  // block per subdomain when it fits in 256 threads, else a cluster of
  // blocks, else the block kernel with up to 1024 threads; FP64 -> block,
  // else (subdomains too large for one block) a cluster of blocks.
  // a warm start (u0) is read by the one-warp and block kernels (and the
  // mapped kernel above); route it to those
  if (u0) {
    a.u0 = u0;
    hz_status ws = HZ_ERR_UNSUPPORTED;
    // the kernel the autotuner chose for this shape when it reads the start
    // (register-resident 1/2/4 warps or block), HZ_SWEEP_WARPS forcing the
    // register-resident shape (tests); else one warp, else the block kernel
    Choice tc{};
    const bool tuned = pr.autotune && lookup_choice(tune_key(pr.g, precision), &tc) &&
                       (tc.variant == kVariantWarp || tc.variant == kVariantBlock);
    const char* hw = std::getenv("HZ_SWEEP_WARPS");
    if (fp32 && !trial && (hw || (tuned && tc.variant == kVariantWarp) || !tuned)) {
      const int h = hw ? std::atoi(hw) : (tuned ? tc.ty : 1);
      ws = launch_choice(pr, a, Choice{kVariantWarp, h}, fp32, st);
      if (ws != HZ_OK && ws != HZ_ERR_UNSUPPORTED) return ws;
      if (ws == HZ_ERR_UNSUPPORTED && h != 1) {
        ws = launch_choice(pr, a, Choice{kVariantWarp, 1}, fp32, st);
        if (ws != HZ_OK && ws != HZ_ERR_UNSUPPORTED) return ws;
      }
    }
    if (ws == HZ_ERR_UNSUPPORTED && tuned && tc.variant == kVariantBlock) {
      ws = launch_choice(pr, a, tc, fp32, st);
      if (ws != HZ_OK && ws != HZ_ERR_UNSUPPORTED) return ws;
    }
    if (ws == HZ_ERR_UNSUPPORTED) HZ_TRY(launch_choice(pr, a, Choice{kVariantBlock, 0}, fp32, st));
    if (e1) HZ_CUDA(cudaEventRecord(e1, st));
    pr.sweeps_launched++;
    return HZ_OK;
  }
  const int want = trial ? kVariantBlock : sweep_variant();  // 16-bit trials run on the block kernel
  Choice ch{};
  bool have = false;
  if (want == kVariantAuto && pr.autotune && lookup_choice(tune_key(pr.g, precision), &ch)) have = true;
  (void)trial;
  hz_status ls = HZ_ERR_UNSUPPORTED;
  if (have) {
    ls = launch_choice(pr, a, ch, fp32, st);
    if (ls != HZ_OK && ls != HZ_ERR_UNSUPPORTED) return ls;
  }
  if (ls == HZ_ERR_UNSUPPORTED && fp32 && (want == kVariantAuto || want == kVariantWarp)) {
    // HZ_SWEEP_WARPS=2|4 forces warps per subdomain of the register-resident kernel (tests)
    const char* hw = std::getenv("HZ_SWEEP_WARPS");
    const int h = hw ? std::atoi(hw) : 1;
    ls = launch_choice(pr, a, Choice{kVariantWarp, h}, fp32, st);
    if (ls != HZ_OK && ls != HZ_ERR_UNSUPPORTED) return ls;
    if (ls != HZ_OK && want == kVariantWarp) return fail(HZ_ERR_UNSUPPORTED, "no warp sweep variant for this subdomain");
  }
  const bool small_block = (int64_t)g.nlx * ((g.nly + g.P - 1) / g.P) <= 256;
  if (ls == HZ_ERR_UNSUPPORTED && fp32 && want == kVariantClusterBand) {  // else only when autotuned
    // HZ_CBAND_ROWS=8 forces 8-row warp bands (tests)
    const char* cr = std::getenv("HZ_CBAND_ROWS");
    ls = launch_choice(pr, a, Choice{kVariantClusterBand, cr ? std::atoi(cr) : 0}, fp32, st);
    if (ls != HZ_OK && ls != HZ_ERR_UNSUPPORTED) return ls;
    if (ls != HZ_OK && want == kVariantClusterBand)
      return fail(HZ_ERR_UNSUPPORTED, "no cluster-of-bands sweep shape fits");
  }
  if (ls == HZ_ERR_UNSUPPORTED && !trial &&
      (want == kVariantCluster || (fp32 && want == kVariantAuto && !small_block))) {
    // HZ_CLUSTER_TY=4 forces 4P rows per thread in the cluster kernel (tests)
    const char* cty = std::getenv("HZ_CLUSTER_TY");
    ls = launch_choice(pr, a, Choice{kVariantCluster, cty ? std::atoi(cty) : 0}, fp32, st);
    if (ls != HZ_OK && ls != HZ_ERR_UNSUPPORTED) return ls;
    if (ls != HZ_OK && want == kVariantCluster) return fail(HZ_ERR_UNSUPPORTED, "no cluster sweep shape fits");
  }
  if (ls == HZ_ERR_UNSUPPORTED) {
    ls = launch_choice(pr, a, Choice{kVariantBlock, 0}, fp32, st);
    // FP64 (and FP32 forced off the cluster heuristic): subdomains too large
    // for one block run on a cluster of blocks
    if (ls == HZ_ERR_UNSUPPORTED && !trial) {
      const char* cty = std::getenv("HZ_CLUSTER_TY");
      const hz_status cs = launch_choice(pr, a, Choice{kVariantCluster, cty ? std::atoi(cty) : 0}, fp32, st);
      if (cs != HZ_ERR_UNSUPPORTED) ls = cs;
    }
    HZ_TRY(ls);
  }
  if (e1) HZ_CUDA(cudaEventRecord(e1, st));
  pr.sweeps_launched++;
  return HZ_OK;
}

static MappedGlobalArgs mapped_args(const Problem& pr) {
  const Geom& g = pr.g;
  MappedGlobalArgs a{};
  a.NXg = g.NXg;
  a.NYg = g.NYg;
  a.nx = g.nx;
  a.ny = g.ny;
  a.P = g.P;
  a.omega = pr.omega;
  for (size_t k = 0; k < pr.mapped_D.size(); ++k) a.D[k] = pr.mapped_D[k];
  a.c = pr.c.as<double>();
  a.geo = pr.mgeog.as<double>();
  a.W = pr.mWg.as<double>();
  a.Hw = pr.mHw.as<double>();
  a.bw = pr.mbw.as<double>();
  a.flux = pr.mflux.as<double>();
  return a;
}

hz_status residual(Problem& pr, const double* b, const double* u, double* r, double* norms2_dev, cudaStream_t st) {
  HZ_TRY(check_ready(pr));
  if (pr.mapped) {
    const MappedGlobalArgs ma = mapped_args(pr);
    HZ_TRY(pr.part.ensure((size_t)std::max(residual_mapped_blocks(ma), 1) * 2 * sizeof(double)));
    int used = 0;
    HZ_TRY(launch_residual_mapped(ma, b, u, r, pr.part.as<double>(), &used, st));
    if (norms2_dev) HZ_TRY(launch_reduce_partials(pr.part.as<double>(), used, 2, norms2_dev, st));
    return HZ_OK;
  }
  const GlobalArgs a = global_args(pr);
  const int nb = residual_blocks(a);
  HZ_TRY(pr.part.ensure((size_t)std::max(nb, 1) * 2 * sizeof(double)));
  int used = 0;
  HZ_TRY(launch_residual(a, b, u, r, pr.part.as<double>(), &used, st));
  if (norms2_dev) HZ_TRY(launch_reduce_partials(pr.part.as<double>(), used, 2, norms2_dev, st));
  return HZ_OK;
}

hz_status rhs(Problem& pr, double* b, cudaStream_t st) {
  HZ_TRY(check_ready(pr));
  if (pr.mapped) return launch_rhs_mapped(mapped_args(pr), pr.f.as<double>(), pr.gb.as<double>(), b, st);
  const GlobalArgs a = global_args(pr);
  return launch_rhs(a, pr.f.as<double>(), pr.gb.as<double>(), b, st);
}

hz_status assemble_add(Problem& pr, const double* u_sub, double* u, cudaStream_t st) {
  const Geom& g = pr.g;
  AssembleArgs a{};
  a.nlx = g.nlx;
  a.nly = g.nly;
  a.Sx = g.Sx;
  a.Sy = g.Sy;
  a.NXg = g.NXg;
  a.NYg = g.NYg;
  a.snxP = g.snx * g.P;
  a.snyP = g.sny * g.P;
  a.share = pr.mapped ? pr.mshare.as<double>() : nullptr;
  return launch_assemble_add(a, u_sub, u, st);
}

// ------------------------------------------------------- outer iteration ----
namespace {

using cplx = std::complex<double>;
constexpr double kGrowthLimit = 1e8;      // see the GMRES loop
constexpr double kResidualGrowth = 1e4;   // refinement step that multiplies the residual by this diverged

struct Ctx {
  Problem& pr;
  const hz_solve_opts& o;
  int nt;
  cudaStream_t st;
  hz_solve_report& rep;
  int64_t n2;  // doubles in a lambda vector
};

// Reads nd doubles from device small-buffer offset 0 and the flag words.
hz_status fetch(Ctx& c, int nd, double* host, int* flags_host) {
  Problem& pr = c.pr;
  HZ_CUDA(cudaMemcpyAsync(pr.hsmall.ptr, pr.small.ptr, (size_t)nd * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  HZ_CUDA(cudaMemcpyAsync(static_cast<char*>(pr.hsmall.ptr) + 4096 * sizeof(double), pr.flags.ptr, 16,
                          cudaMemcpyDeviceToHost, c.st));
  HZ_CUDA(cudaStreamSynchronize(c.st));
  std::memcpy(host, pr.hsmall.ptr, (size_t)nd * sizeof(double));
  std::memcpy(flags_host, static_cast<char*>(pr.hsmall.ptr) + 4096 * sizeof(double), 16);
  if (flags_host[0] & 1) return fail(HZ_ERR_DIVERGED, "non-finite values in the subdomain solve (time step too large?)");
  for (int k = 0; k < nd; ++k)
    if (!std::isfinite(host[k])) return fail(HZ_ERR_DIVERGED, "non-finite value in the outer iteration");
  return HZ_OK;
}

// out[0..2nv) = reduced dots of V_0..V_{nv-1} with w, or with w - w_sub
// (then also written to w_out).
hz_status dots_to(Ctx& c, const double* V, int64_t ld, int nv, const double* w, bool real, double* out,
                  const double* w_sub = nullptr, double* w_out = nullptr) {
  Problem& pr = c.pr;
  const int nb = vec_blocks(c.n2);
  HZ_TRY(pr.part.ensure((size_t)nb * nv * 2 * sizeof(double) + 64));
  HZ_TRY(launch_multi_dot(V, ld, nv, w, w_sub, w_out, c.n2, real, pr.part.as<double>(), nb, c.st));
  return launch_reduce_partials(pr.part.as<double>(), nb, 2 * nv, out, c.st);
}

hz_status dots(Ctx& c, const double* V, int64_t ld, int nv, const double* w, bool real, int off) {
  return dots_to(c, V, ld, nv, w, real, c.pr.small.as<double>() + off);
}

// Outer-iteration sweeps keep one sweep of the budget in reserve for the
// closing sweep of the DD solve (reserve = 1); the closing sweep uses 0.
hz_status do_sweep(Ctx& c, const double* lam_in, double* lam_out, const double* rhs, double* u_sub, int reserve = 1,
                   const double* u0 = nullptr) {
  if (c.rep.sweeps + reserve >= c.o.max_sweeps) return fail(HZ_ERR_NOT_CONVERGED, "sweep budget exhausted");
  HZ_TRY(sweep(c.pr, c.o.precision, c.nt, c.o.wh_iters, c.o.wh_tol, lam_in, lam_out, rhs, u_sub, c.st, u0));
  c.rep.sweeps++;
  return HZ_OK;
}

// Approximate K^{-1} rhs by the DD method and add it to u.
hz_status dd_solve(Ctx& c, const double* rhs, double* u) {
  Problem& pr = c.pr;
  const Geom& g = pr.g;
  const int64_t n2 = c.n2;
  const size_t vb = (size_t)n2 * sizeof(double);
  const int m = std::max(1, c.o.gmres_restart);
  const bool real = c.o.outer == HZ_OUTER_RGMRES;
  HZ_TRY(pr.gv.ensure(vb));
  HZ_TRY(pr.xv.ensure(vb));
  HZ_TRY(pr.tv.ensure(vb));
  HZ_TRY(pr.usub.ensure((size_t)g.L * g.sub_nodes() * 2 * sizeof(double)));
  HZ_TRY(pr.small.ensure(8192 * sizeof(double)));
  HZ_TRY(pr.hsmall.ensure(8192 * sizeof(double)));
  double* gv = pr.gv.as<double>();
  double* xv = pr.xv.as<double>();
  double* tv = pr.tv.as<double>();
  HZ_CUDA(cudaMemsetAsync(xv, 0, vb, c.st));
  // g = T(0): sweep with zero transmission data and the source
  // warm start (plain iteration): every sweep's WaveHoltz starts from the
  // previous sweep's subdomain solutions, carried in uwarm (in place: each
  // subdomain reads its start at the beginning of the sweep and writes its
  // result at the end)
  const bool warm = c.o.wh_warm && c.o.outer == HZ_OUTER_PLAIN;
  double* uw = nullptr;
  if (warm) {
    HZ_TRY(pr.uwarm.ensure((size_t)g.L * g.sub_nodes() * 2 * sizeof(double)));
    uw = pr.uwarm.as<double>();
  }
  HZ_TRY(do_sweep(c, xv, gv, rhs, uw));
  int flags[4];
  double hbuf[8192];
  HZ_TRY(dots(c, gv, 0, 1, gv, real, 0));
  HZ_TRY(fetch(c, 2, hbuf, flags));
  const double gnorm = std::sqrt(hbuf[0]);
  const double tol = c.o.inner_tol;
  if (gnorm > 0.0) {
    if (c.o.outer == HZ_OUTER_PLAIN) {
      // lambda <- S(lambda) + g, i.e. a sweep with the source (eq. (lambda-iteration))
      HZ_CUDA(cudaMemcpyAsync(xv, gv, vb, cudaMemcpyDeviceToDevice, c.st));
      while (true) {
        hz_status s = do_sweep(c, xv, tv, rhs, uw, 1, uw);
        if (s == HZ_ERR_NOT_CONVERGED) break;
        HZ_TRY(s);
        HZ_TRY(launch_axpby(1.0, tv, -1.0, xv, n2, c.st));  // xv = tv - xv (difference)
        HZ_TRY(dots(c, xv, 0, 1, xv, true, 0));
        HZ_TRY(fetch(c, 2, hbuf, flags));
        if (!(std::sqrt(hbuf[0]) < kGrowthLimit * gnorm))
          return fail(HZ_ERR_DIVERGED, "fixed-point iteration exploded: time step beyond the stability limit?");
        HZ_CUDA(cudaMemcpyAsync(xv, tv, vb, cudaMemcpyDeviceToDevice, c.st));
        c.rep.gmres_iters++;
        if (std::sqrt(hbuf[0]) <= tol * gnorm) break;
      }
    } else {
      HZ_TRY(pr.V.ensure(vb * (m + 1)));
      double* V = pr.V.as<double>();
      std::vector<cplx> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1);
      bool first = true, done = false;
      while (!done) {
        // residual of the current iterate into V_0
        if (first) {
          HZ_CUDA(cudaMemcpyAsync(V, gv, vb, cudaMemcpyDeviceToDevice, c.st));
          first = false;
        } else {
          hz_status s = do_sweep(c, xv, tv, nullptr, nullptr);
          if (s == HZ_ERR_NOT_CONVERGED) break;
          HZ_TRY(s);
          // V0 = g - (x - S x) = g - x + t
          HZ_CUDA(cudaMemcpyAsync(V, gv, vb, cudaMemcpyDeviceToDevice, c.st));
          HZ_TRY(launch_axpby(-1.0, xv, 1.0, V, n2, c.st));
          HZ_TRY(launch_axpby(1.0, tv, 1.0, V, n2, c.st));
        }
        HZ_TRY(dots(c, V, 0, 1, V, real, 0));
        HZ_TRY(fetch(c, 2, hbuf, flags));
        const double beta = std::sqrt(hbuf[0]);
        if (beta <= tol * gnorm) break;
        HZ_TRY(launch_axpby(0.0, V, 1.0 / beta, V, n2, c.st));
        std::fill(gvec.begin(), gvec.end(), cplx(0.0));
        gvec[0] = beta;
        int k = 0;
        // Pipelined Arnoldi: step j's device work (sweep, two classical
        // Gram-Schmidt passes, norm, normalisation of V_{j+1} by a device-side
        // 1/||w||) needs nothing from the host, so step j+1 is enqueued before
        // the host waits for column j of the Hessenberg matrix; the host's
        // Givens update overlaps the next sweep.  A converged cycle leaves one
        // enqueued step unused.
        const size_t CS = (size_t)4 * m + 8;  // per column: pass-1 dots (m+2), pass-2 dots (m+1), norm: complex
        const size_t CS2 = CS + 2;            // + the 4 status words (16 bytes), read back with the column
        HZ_TRY(pr.hcol.ensure((size_t)(m + 1) * CS2 * sizeof(double)));
        HZ_TRY(pr.hcol_host.ensure((size_t)(m + 1) * (CS + 4) * sizeof(double)));
        while (pr.gm_events.size() < (size_t)(m + 1)) {
          cudaEvent_t e;
          HZ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
          pr.gm_events.push_back(e);
        }
        double* hd = pr.hcol.as<double>();
        double* hh = pr.hcol_host.as<double>();
        // the step's vector work after its sweep (a fixed sequence of launches
        // for a given j: captured as a CUDA graph with opts.graphs):
        // w = v_j - S v_j with the pass-1 dots, pass-1 update, [pass-2 dots,
        // pass-2 update,] the last update with ||w||^2, normalisation
        const bool two_pass = c.o.gs_passes == 2;
        auto post = [&](int j) -> hz_status {
          double* vj = V + (size_t)j * n2;
          double* w = V + (size_t)(j + 1) * n2;
          const int nv = j + 1;
          double* col = hd + (size_t)j * CS2;
          double* nrm = col + 2 * (m + 2) + 2 * (m + 1);
          HZ_TRY(dots_to(c, V, n2, nv, vj, real, col, tv, w));
          if (two_pass) {
            HZ_TRY(launch_multi_axpy(V, n2, nv, col, w, n2, real, c.st));
            HZ_TRY(dots_to(c, V, n2, nv, w, real, col + 2 * (m + 2)));
          }
          HZ_TRY(launch_multi_axpy(V, n2, nv, two_pass ? col + 2 * (m + 2) : col, w, n2, real, c.st,
                                   pr.part.as<double>()));
          HZ_TRY(launch_reduce_partials(pr.part.as<double>(), axpy_blocks(n2), 2, nrm, c.st));
          HZ_TRY(launch_scale_inv_norm(w, nrm, w, n2, c.st, pr.flags.as<int>(), reinterpret_cast<int*>(col + CS)));
          double* hslot = hh + (size_t)j * (CS + 4);
          HZ_CUDA(cudaMemcpyAsync(hslot, col, CS2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
          // while a graph is captured the record must be external to become an
          // event node the host can wait on
          cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
          HZ_CUDA(cudaStreamIsCapturing(c.st, &cap));
          if (cap == cudaStreamCaptureStatusActive)
            HZ_CUDA(cudaEventRecordWithFlags(pr.gm_events[j], c.st, cudaEventRecordExternal));
          else
            HZ_CUDA(cudaEventRecord(pr.gm_events[j], c.st));
          return HZ_OK;
        };
        const bool graphs = c.o.graphs && !is_default_stream(c.st);  // default streams cannot be captured
        // partials of the dots (up to m + 1 vectors) and of the norm; allocated
        // before any step (and before a capture, which must not allocate)
        HZ_TRY(pr.part.ensure((size_t)std::max(vec_blocks(n2) * (m + 1), axpy_blocks(n2)) * 2 * sizeof(double) + 64));
        if (graphs) {
          const std::vector<const void*> key = {V, tv, hd, hh, pr.flags.ptr, pr.part.ptr, (const void*)(intptr_t)n2,
                                                (const void*)(intptr_t)m, (const void*)(intptr_t)real,
                                                (const void*)(intptr_t)two_pass};
          if (key != pr.step_graph_key) {
            release_step_graphs(pr);
            pr.step_graph_key = key;
          }
          if ((int)pr.step_graphs.size() < m) {
            pr.step_graphs.resize(m, nullptr);
            pr.step_graph_kernels.resize(m, 0);
          }
        }
        auto enqueue = [&](int j) -> hz_status {
          hz_status s = do_sweep(c, V + (size_t)j * n2, tv, nullptr, nullptr);
          if (s != HZ_OK) return s;
          if (!graphs) return post(j);
          if (!pr.step_graphs[j]) {
            const unsigned long long k0 = launch_count();
            HZ_CUDA(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal));
            const hz_status ps = post(j);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(c.st, &graph);
            const long long kn = (long long)(launch_count() - k0);
            add_launches(-kn);  // counted when the graph runs
            if (ps != HZ_OK || ce != cudaSuccess) {
              if (graph) cudaGraphDestroy(graph);
              (void)cudaGetLastError();
              return ps != HZ_OK ? ps : cuda_fail(ce, "capture of the Arnoldi step");
            }
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
            pr.step_graphs[j] = ex;
            pr.step_graph_kernels[j] = kn;
          }
          HZ_CUDA(cudaGraphLaunch(pr.step_graphs[j], c.st));
          add_launches(pr.step_graph_kernels[j]);
          return HZ_OK;
        };
        hz_status es = enqueue(0);
        if (es == HZ_ERR_NOT_CONVERGED) break;
        HZ_TRY(es);
        for (int j = 0; j < m; ++j) {
          bool next = false;
          if (j + 1 < m) {
            es = enqueue(j + 1);
            if (es == HZ_OK) next = true;
            else if (es != HZ_ERR_NOT_CONVERGED) return es;
          }
          HZ_CUDA(cudaEventSynchronize(pr.gm_events[j]));
          const double* hslot = hh + (size_t)j * (CS + 4);
          int fl[4];
          std::memcpy(fl, hslot + CS, 16);
          if (fl[0] & 1) return fail(HZ_ERR_DIVERGED, "non-finite values in the subdomain solve (time step too large?)");
          c.rep.gmres_iters++;
          for (int i = 0; i <= j; ++i)
            H[(size_t)i * m + j] = two_pass ? cplx(hslot[2 * i] + hslot[2 * (m + 2) + 2 * i],
                                                   hslot[2 * i + 1] + hslot[2 * (m + 2) + 2 * i + 1])
                                            : cplx(hslot[2 * i], hslot[2 * i + 1]);
          const double hn2 = hslot[2 * (m + 2) + 2 * (m + 1)];
          const double hnext = std::sqrt(std::max(0.0, hn2));
          // ||(I - S) v|| for a unit v is O(1) for a stable subdomain solve; growth by
          // many orders of magnitude means the leapfrog is unstable (time step too large)
          if (!(hnext < kGrowthLimit) || !(std::abs(H[(size_t)j * m + j]) < kGrowthLimit))
            return fail(HZ_ERR_DIVERGED, "sweep operator norm exploded: time step beyond the stability limit?");
          // apply previous rotations
          for (int i = 0; i < j; ++i) {
            const cplx a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
            H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
            H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * b;
          }
          const cplx a = H[(size_t)j * m + j];
          const double rr = std::sqrt(std::norm(a) + hnext * hnext);
          if (std::abs(a) == 0.0) {
            cs[j] = 0.0;
            sn[j] = 1.0;
          } else {
            cs[j] = std::abs(a) / rr;
            sn[j] = (a / std::abs(a)) * hnext / rr;
          }
          H[(size_t)j * m + j] = cs[j] * a + sn[j] * hnext;
          gvec[j + 1] = -std::conj(sn[j]) * gvec[j];
          gvec[j] = cs[j] * gvec[j];
          k = j + 1;
          const double res = std::abs(gvec[j + 1]);
          if (res <= tol * gnorm || hnext == 0.0) { done = true; break; }
          if (!next) {
            if (j + 1 < m) done = true;  // sweep budget exhausted
            break;
          }
        }
        if (k > 0) {
          // back substitution R y = gvec, then x += V y  (multi_axpy subtracts, so pass -y)
          std::vector<cplx> y(k);
          for (int i = k - 1; i >= 0; --i) {
            cplx s = gvec[i];
            for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
            y[i] = s / H[(size_t)i * m + i];
          }
          std::vector<double> ny(2 * k);
          for (int i = 0; i < k; ++i) {
            ny[2 * i] = -y[i].real();
            ny[2 * i + 1] = real ? 0.0 : -y[i].imag();
          }
          HZ_CUDA(cudaMemcpyAsync(pr.small.ptr, ny.data(), ny.size() * sizeof(double), cudaMemcpyHostToDevice, c.st));
          HZ_TRY(launch_multi_axpy(V, n2, k, pr.small.as<double>(), xv, n2, real, c.st));
          HZ_CUDA(cudaStreamSynchronize(c.st));  // ny leaves scope
        }
      }
    }
  }
  // final sweep at the converged transmission data: subdomain solutions -> u
  hz_solve_opts relaxed = c.o;
  relaxed.max_sweeps = std::max(c.o.max_sweeps, c.rep.sweeps + 1);  // the closing sweep is always allowed
  Ctx cf{pr, relaxed, c.nt, c.st, c.rep, c.n2};
  HZ_TRY(do_sweep(cf, xv, tv, rhs, pr.usub.as<double>(), 0, uw));
  HZ_TRY(assemble_add(pr, pr.usub.as<double>(), u, c.st));
  return HZ_OK;
}

// FP64 flexible GMRES on the global system K u = b, right-preconditioned by
// the DD solve (Sec. 7: the DD cycle is a preconditioner and may run in
// lower precision).  Krylov step j applies the preconditioner, z_j = DD(v_j)
// -- one outer iteration on the transmission data with FP32 (or FP64)
// sweeps, to inner_tol -- and the global operator, w = K z_j, then two
// passes of classical Gram-Schmidt on the global vectors.  The z_j are kept
// because the preconditioner changes from step to step (WaveHoltz with a
// fixed count is only real-linear, and the inner GMRES stops at a
// tolerance); u += Z y with y minimising ||beta e1 - H y||.  Every cycle
// restarts from the true FP64 residual.  Plain defect correction takes the
// last correction alone; when the FP32 preconditioner is accurate to only a
// fraction in a few ill-conditioned directions, that stagnates, while the
// minimisation over all corrections of a cycle removes those directions.
// rep.refinements counts preconditioner applications.
hz_status fgmres_refine(Ctx& c, double* u, hz_status* result) {
  Problem& pr = c.pr;
  const Geom& g = pr.g;
  const hz_solve_opts& o = c.o;
  const int64_t n2 = 2 * g.n;
  const size_t vb = (size_t)n2 * sizeof(double);
  const int m = std::max(1, std::min(o.refine_restart, 200));
  HZ_TRY(pr.Vg.ensure(vb * (m + 1)));
  HZ_TRY(pr.Zg.ensure(vb * m));
  double* V = pr.Vg.as<double>();
  double* Z = pr.Zg.as<double>();
  Ctx cv{pr, o, c.nt, c.st, c.rep, n2};  // vector work on global vectors
  HZ_TRY(pr.part.ensure((size_t)std::max(vec_blocks(n2) * (m + 1), axpy_blocks(n2)) * 2 * sizeof(double) + 64));
  std::vector<cplx> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1);
  std::vector<double> hb(4 * (size_t)m + 16);
  int flags[4];
  double* sm = pr.small.as<double>();
  while (true) {
    // r = b - K u into V_0, with ||r||^2 and ||b||^2
    HZ_TRY(residual(pr, pr.bvec.as<double>(), u, V, sm, c.st));
    HZ_TRY(fetch(c, 2, hb.data(), flags));
    const double bnorm = std::sqrt(hb[1]);
    const double beta = std::sqrt(hb[0]);
    const double rel = bnorm > 0.0 ? beta / bnorm : 0.0;
    // a cycle's update that multiplied the true residual (or made it
    // non-finite: a singular least-squares system) diverged
    if (!std::isfinite(rel) || (c.rep.refinements > 0 && !(rel < kResidualGrowth * c.rep.rel_residual))) {
      c.rep.rel_residual = rel;
      return fail(HZ_ERR_DIVERGED, "refinement cycle increased the residual by orders of magnitude");
    }
    c.rep.rel_residual = rel;
    if (rel <= o.tol) {
      *result = HZ_OK;
      return HZ_OK;
    }
    if (c.rep.refinements >= o.max_refine || c.rep.sweeps + 2 > o.max_sweeps) {
      *result = fail(HZ_ERR_NOT_CONVERGED, "tolerance not reached within the refinement / sweep budget");
      return HZ_OK;
    }
    HZ_TRY(launch_axpby(0.0, V, 1.0 / beta, V, n2, c.st));
    std::fill(gvec.begin(), gvec.end(), cplx(0.0));
    gvec[0] = beta;
    int k = 0;
    double est = rel;
    for (int j = 0; j < m; ++j) {
      if (c.rep.refinements >= o.max_refine || c.rep.sweeps + 2 > o.max_sweeps) break;
      double* vj = V + (size_t)j * n2;
      double* zj = Z + (size_t)j * n2;
      double* w = V + (size_t)(j + 1) * n2;
      // z_j = DD(v_j)
      HZ_CUDA(cudaMemsetAsync(zj, 0, vb, c.st));
      hz_solve_opts oi = o;
      if (o.wh_adaptive) oi.wh_tol = std::min(1e-2, std::max(o.wh_tol > 0.0 ? o.wh_tol : 1e-6, 0.1 * est));
      Ctx ci{pr, oi, c.nt, c.st, c.rep, c.n2};
      const hz_status ds = dd_solve(ci, vj, zj);
      if (ds != HZ_OK && ds != HZ_ERR_NOT_CONVERGED) return ds;
      c.rep.refinements++;
      // w = K z_j (the residual kernel with b = 0 gives -K z_j)
      HZ_TRY(residual(pr, nullptr, zj, w, nullptr, c.st));
      HZ_TRY(launch_axpby(0.0, w, -1.0, w, n2, c.st));
      // two passes of classical Gram-Schmidt, then ||w||
      const int nv = j + 1;
      HZ_TRY(dots_to(cv, V, n2, nv, w, false, sm));
      HZ_TRY(launch_multi_axpy(V, n2, nv, sm, w, n2, false, c.st));
      HZ_TRY(dots_to(cv, V, n2, nv, w, false, sm + 2 * nv));
      HZ_TRY(launch_multi_axpy(V, n2, nv, sm + 2 * nv, w, n2, false, c.st));
      HZ_TRY(dots_to(cv, w, 0, 1, w, false, sm + 4 * nv));
      HZ_TRY(fetch(c, 4 * nv + 2, hb.data(), flags));
      for (int i = 0; i <= j; ++i)
        H[(size_t)i * m + j] = cplx(hb[2 * i] + hb[2 * nv + 2 * i], hb[2 * i + 1] + hb[2 * nv + 2 * i + 1]);
      const double hnext = std::sqrt(std::max(0.0, hb[4 * nv]));
      if (!(hnext < kGrowthLimit * std::max(1.0, bnorm)) || !std::isfinite(std::abs(H[(size_t)j * m + j])))
        return fail(HZ_ERR_DIVERGED, "refinement Krylov step exploded: time step beyond the stability limit?");
      if (hnext > 0.0) HZ_TRY(launch_axpby(0.0, w, 1.0 / hnext, w, n2, c.st));
      for (int i = 0; i < j; ++i) {
        const cplx a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -std::conj(sn[i]) * a + cs[i] * b;
      }
      const cplx a = H[(size_t)j * m + j];
      const double rr = std::sqrt(std::norm(a) + hnext * hnext);
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = std::abs(a) / rr;
        sn[j] = (a / std::abs(a)) * hnext / rr;
      }
      H[(size_t)j * m + j] = cs[j] * a + sn[j] * hnext;
      gvec[j + 1] = -std::conj(sn[j]) * gvec[j];
      gvec[j] = cs[j] * gvec[j];
      k = j + 1;
      est = bnorm > 0.0 ? std::abs(gvec[j + 1]) / bnorm : 0.0;
      if (std::getenv("HZ_SOLVE_LOG"))  // progress of long solves (diagnostics)
        std::fprintf(stderr, "hz fgmres: DD solve %d, sweeps %d, residual estimate %.3e\n", c.rep.refinements,
                     c.rep.sweeps, est);
      if (est <= 0.5 * o.tol || hnext == 0.0) break;
    }
    if (k == 0) {
      *result = fail(HZ_ERR_NOT_CONVERGED, "tolerance not reached within the refinement / sweep budget");
      return HZ_OK;
    }
    // y from the triangular system, then u += Z y (multi_axpy subtracts: pass -y)
    std::vector<cplx> y(k);
    for (int i = k - 1; i >= 0; --i) {
      cplx s = gvec[i];
      for (int q = i + 1; q < k; ++q) s -= H[(size_t)i * m + q] * y[q];
      y[i] = s / H[(size_t)i * m + i];
    }
    double* ny = pr.hsmall.as<double>();
    for (int i = 0; i < k; ++i) {
      ny[2 * i] = -y[i].real();
      ny[2 * i + 1] = -y[i].imag();
    }
    HZ_CUDA(cudaMemcpyAsync(sm, ny, (size_t)2 * k * sizeof(double), cudaMemcpyHostToDevice, c.st));
    HZ_TRY(launch_multi_axpy(Z, n2, k, sm, u, n2, false, c.st));
    HZ_CUDA(cudaStreamSynchronize(c.st));  // the pinned staging buffer is reused
  }
}

}  // namespace

hz_solve_opts effective_opts(const hz_solve_opts& o) {
  hz_solve_opts e = o;
  if (e.wh_iters == 0 && e.wh_tol > 0.0) e.wh_iters = kDefaultWhCap;
  return e;
}

hz_status solve(Problem& pr, const hz_solve_opts& o_in, double* u, hz_solve_report* rep_out, cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  const hz_solve_opts o = effective_opts(o_in);
  HZ_TRY(check_ready(pr));
  if (!(o.tol >= 0.0) || o.max_sweeps < 1 || o.gmres_restart < 1 || o.gmres_restart > 1000 || o.wh_iters < 1 ||
      !(o.cfl > 0.0) || o.max_refine < 0 || !(o.inner_tol >= 0.0) || !(o.wh_tol >= 0.0))
    return fail(HZ_ERR_INVALID_ARG, "invalid solve options");
  if (o.outer < HZ_OUTER_GMRES || o.outer > HZ_OUTER_RGMRES) return fail(HZ_ERR_INVALID_ARG, "unknown outer");
  if (o.gs_passes != 1 && o.gs_passes != 2) return fail(HZ_ERR_INVALID_ARG, "gs_passes must be 1 or 2");
  if (o.refine != HZ_REFINE_DEFECT && o.refine != HZ_REFINE_FGMRES)
    return fail(HZ_ERR_INVALID_ARG, "unknown refinement");
  if (o.refine == HZ_REFINE_FGMRES && (o.refine_restart < 1 || o.refine_restart > 200))
    return fail(HZ_ERR_INVALID_ARG, "refine_restart must be in 1..200");
  if (o.wh_warm != 0 && (o.wh_warm != 1 || o.outer != HZ_OUTER_PLAIN))
    return fail(HZ_ERR_INVALID_ARG, "wh_warm = 1 needs the plain outer iteration (GMRES needs a fixed linear sweep)");
  hz_solve_report rep{};
  const int nt = o.nt_override > 0 ? o.nt_override : choose_nt(pr, o.cfl);
  rep.nt = nt;
  const Geom& g = pr.g;
  const size_t nb = (size_t)g.n * 2 * sizeof(double);
  HZ_TRY(pr.bvec.ensure(nb));
  HZ_TRY(pr.rvec.ensure(nb));
  HZ_TRY(pr.small.ensure(8192 * sizeof(double)));
  HZ_TRY(pr.hsmall.ensure(8192 * sizeof(double)));
  HZ_TRY(prepare(pr, nt, st));
  HZ_TRY(ensure_flags(pr));
  pr.autotune = o.autotune != 0 && sweep_variant() == kVariantAuto && o.precision <= HZ_FP32_REFINE && !pr.mapped;
  if (pr.autotune) HZ_TRY(autotune(pr, o.precision, nt, o.wh_iters, st));
  HZ_CUDA(cudaMemsetAsync(pr.flags.ptr, 0, 64, st));
  HZ_TRY(rhs(pr, pr.bvec.as<double>(), st));
  HZ_CUDA(cudaMemsetAsync(u, 0, nb, st));
  Ctx c{pr, o, nt, st, rep, 2 * g.lam_complex()};
  pr.time_sweeps = true;
  pr.ev_used = 0;
  struct TimingOff {  // direct hz_sweep calls after a failed solve record nothing
    Problem& p;
    ~TimingOff() { p.time_sweeps = false; }
  } timing_off{pr};
  double hb[4];
  int flags[4];
  hz_status result = HZ_OK;
  double bnorm = 0.0;
  if (o.refine == HZ_REFINE_FGMRES) {
    const hz_status fs = fgmres_refine(c, u, &result);
    if (fs != HZ_OK) {
      if (rep_out) *rep_out = rep;
      return fs;
    }
  }
  while (o.refine != HZ_REFINE_FGMRES) {
    HZ_TRY(residual(pr, pr.bvec.as<double>(), u, pr.rvec.as<double>(), pr.small.as<double>(), st));
    HZ_TRY(fetch(c, 2, hb, flags));
    bnorm = std::sqrt(hb[1]);
    const double rel = bnorm > 0.0 ? std::sqrt(hb[0]) / bnorm : 0.0;
    if (rep.refinements > 0 && !(rel < kResidualGrowth * rep.rel_residual)) {
      rep.rel_residual = rel;
      if (rep_out) *rep_out = rep;
      return fail(HZ_ERR_DIVERGED, "refinement step increased the residual by orders of magnitude");
    }
    rep.rel_residual = rel;
    if (std::getenv("HZ_SOLVE_LOG"))
      std::fprintf(stderr, "hz refinement %d: sweeps %d, residual %.3e\n", rep.refinements, rep.sweeps, rel);
    if (rel <= o.tol) break;
    if (rep.refinements >= o.max_refine || rep.sweeps + 2 > o.max_sweeps) {  // a DD solve needs >= 2 sweeps
      result = fail(HZ_ERR_NOT_CONVERGED, "tolerance not reached within the refinement / sweep budget");
      break;
    }
    // variable inner tolerance (Sec. 5 end, Sec. 8): loose subdomain solves while
    // the global residual is large, tightened as it falls
    hz_solve_opts oi = o;
    if (o.wh_adaptive) oi.wh_tol = std::min(1e-2, std::max(o.wh_tol > 0.0 ? o.wh_tol : 1e-6, 0.1 * rel));
    Ctx ci{pr, oi, nt, st, rep, c.n2};
    hz_status s = dd_solve(ci, pr.rvec.as<double>(), u);
    if (s != HZ_OK && s != HZ_ERR_NOT_CONVERGED) {
      if (rep_out) *rep_out = rep;
      return s;
    }
    rep.refinements++;
  }
  HZ_CUDA(cudaMemcpyAsync(flags, pr.flags.ptr, 16, cudaMemcpyDeviceToHost, st));
  HZ_CUDA(cudaStreamSynchronize(st));
  unsigned long long itsum = 0;
  std::memcpy(&itsum, &flags[2], sizeof(itsum));
  rep.wh_iters_max = flags[1];
  rep.dof_updates = (int64_t)itsum * g.sub_nodes() * (nt - 1);
  double sw = 0.0;
  for (size_t k = 0; k + 1 < pr.ev_used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pr.events[k], pr.events[k + 1]) == cudaSuccess) sw += ms * 1e-3;
  }
  (void)cudaGetLastError();
  rep.sweep_seconds = sw;
  rep.sweep_variant = pr.last_variant;
  rep.sweep_shape = pr.last_shape;
  pr.time_sweeps = false;
  rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep_out) *rep_out = rep;
  return result;
}

}  // namespace hz

// =========================================================== C ABI ====
using namespace hz;

namespace {
template <typename F>
hz_status guard(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(HZ_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(HZ_ERR_INTERNAL, e.what());
  } catch (...) {
    return fail(HZ_ERR_INTERNAL, "unknown exception");
  }
}

hz_status use_device(const Problem& pr) {
  HZ_CUDA(cudaSetDevice(pr.device));
  return HZ_OK;
}

bool all_finite(const double* p, int64_t n) {
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

int64_t field_count(const Geom& g, hz_field f) {
  switch (f) {
    case HZ_WAVE_SPEED: return g.n;
    case HZ_OMEGA: return 1;
    case HZ_SOURCE: return g.n;
    case HZ_BOUNDARY: return 2 * (int64_t)g.NXg + 2 * (int64_t)g.NYg;
    case HZ_TRANSMISSION: return 2;
    case HZ_NODE_COORDS: return 2 * g.n;
  }
  return -1;
}

hz_status set_field_host(Problem& pr, hz_field field, const double* data, int64_t count) {
  const Geom& g = pr.g;
  if (!data) return fail(HZ_ERR_INVALID_ARG, "null data");
  const int64_t want = field_count(g, field);
  if (want < 0) return fail(HZ_ERR_INVALID_ARG, "unknown field");
  if (count != want) return fail(HZ_ERR_INVALID_ARG, "wrong value count for field");
  const bool cplx_field = field == HZ_SOURCE || field == HZ_BOUNDARY;
  const int64_t nd = cplx_field ? 2 * count : count;
  if (!all_finite(data, nd)) return fail(HZ_ERR_INVALID_ARG, "non-finite input");
  HZ_TRY(use_device(pr));
  switch (field) {
    case HZ_WAVE_SPEED: {
      double cmax = 0.0;
      for (int64_t k = 0; k < count; ++k) {
        if (!(data[k] > 0.0)) return fail(HZ_ERR_INVALID_ARG, "wave speed must be > 0");
        cmax = std::max(cmax, data[k]);
      }
      HZ_TRY(pr.c.ensure(nd * sizeof(double)));
      HZ_CUDA(cudaMemcpy(pr.c.ptr, data, nd * sizeof(double), cudaMemcpyHostToDevice));
      pr.cmax = cmax;
      pr.has_c = true;
      break;
    }
    case HZ_OMEGA:
      if (!(data[0] > 0.0)) return fail(HZ_ERR_INVALID_ARG, "omega must be > 0");
      pr.omega = data[0];
      pr.has_omega = true;
      break;
    case HZ_SOURCE:
      HZ_TRY(pr.f.ensure(nd * sizeof(double)));
      HZ_CUDA(cudaMemcpy(pr.f.ptr, data, nd * sizeof(double), cudaMemcpyHostToDevice));
      break;
    case HZ_BOUNDARY:
      HZ_TRY(pr.gb.ensure(nd * sizeof(double)));
      HZ_CUDA(cudaMemcpy(pr.gb.ptr, data, nd * sizeof(double), cudaMemcpyHostToDevice));
      break;
    case HZ_TRANSMISSION:
      if (!(data[0] >= 0.0) || !(data[1] > 0.0)) return fail(HZ_ERR_INVALID_ARG, "need eta >= 0 and zeta > 0");
      pr.robin_eta = data[0];
      pr.robin_zeta = data[1];
      break;
    case HZ_NODE_COORDS:
      HZ_TRY(set_node_coords(pr, data));
      break;
  }
  HZ_UPLOADS_DONE();
  pr.version++;
  return HZ_OK;
}

hz_status opts_or_default(const hz_solve_opts* o, hz_solve_opts* out) {
  if (o) *out = *o;
  else hz_default_opts(out);
  return HZ_OK;
}
}  // namespace

extern "C" {

hz_status hz_kernel_launches(uint64_t* count) {
  if (!count) return fail(HZ_ERR_INVALID_ARG, "null argument");
  *count = g_launches.load();
  return HZ_OK;
}

void hz_default_opts(hz_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = HZ_FP64;
  o->tol = 1e-8;
  o->max_sweeps = 2000;
  o->outer = HZ_OUTER_GMRES;
  o->gmres_restart = 60;
  o->wh_iters = 20;
  o->wh_tol = 0.0;
  o->nt_override = 0;
  o->cfl = 0.9;
  o->inner_tol = 1e-2;
  o->max_refine = 20;
  o->autotune = 1;
  o->pack = 1;
  o->graphs = 1;
  o->gs_passes = 1;
  o->refine = HZ_REFINE_DEFECT;
  o->refine_restart = 30;
}

hz_status hz_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return HZ_ERR_INVALID_ARG;
  std::strncpy(buf, g_last_error.c_str(), n - 1);
  buf[n - 1] = '\0';
  return HZ_OK;
}

hz_status hz_mesh_create(double x0, double x1, double y0, double y1, int32_t nx, int32_t ny, int32_t degree,
                         int32_t sub_nx, int32_t sub_ny, hz_mesh* out) {
  return guard([&]() -> hz_status {
    if (!out) return fail(HZ_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    auto* m = new hz_mesh_s();
    hz_status s = build_geom(x0, x1, y0, y1, nx, ny, degree, sub_nx, sub_ny, &m->g);
    if (s != HZ_OK) {
      delete m;
      return s;
    }
    *out = m;
    return HZ_OK;
  });
}

hz_status hz_mesh_num_nodes(hz_mesh mesh, int64_t* n) {
  if (!mesh || !n) return fail(HZ_ERR_INVALID_ARG, "null argument");
  *n = mesh->g.n;
  return HZ_OK;
}

hz_status hz_mesh_node_coords(hz_mesh mesh, double* xy) {
  if (!mesh || !xy) return fail(HZ_ERR_INVALID_ARG, "null argument");
  const Geom& g = mesh->g;
  for (int J = 0; J < g.NYg; ++J) {
    const int ey = std::min(J / g.P, g.ny - 1), b = J - ey * g.P;
    const double y = g.y0 + ey * g.hy + (g.xi[b] + 1.0) * g.hy / 2.0;
    for (int I = 0; I < g.NXg; ++I) {
      const int ex = std::min(I / g.P, g.nx - 1), a = I - ex * g.P;
      const double x = g.x0 + ex * g.hx + (g.xi[a] + 1.0) * g.hx / 2.0;
      xy[2 * ((int64_t)J * g.NXg + I)] = x;
      xy[2 * ((int64_t)J * g.NXg + I) + 1] = y;
    }
  }
  return HZ_OK;
}

void hz_mesh_destroy(hz_mesh mesh) { delete mesh; }

hz_status hz_problem_create(hz_mesh mesh, int32_t device, hz_problem* out) {
  return guard([&]() -> hz_status {
    if (!mesh || !out) return fail(HZ_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    int ndev = 0;
    HZ_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(HZ_ERR_INVALID_ARG, "no such CUDA device");
    auto* pr = new hz_problem_s();
    pr->g = mesh->g;
    pr->device = device;
    hz_status s = [&]() -> hz_status {
      HZ_CUDA(cudaSetDevice(device));
      const Geom& g = pr->g;
      HZ_TRY(pr->Wxg.ensure(g.Wxg.size() * sizeof(double)));
      HZ_TRY(pr->Wyg.ensure(g.Wyg.size() * sizeof(double)));
      HZ_TRY(pr->wxs.ensure(g.Wxs.size() * sizeof(double)));
      HZ_TRY(pr->wys.ensure(g.Wys.size() * sizeof(double)));
      HZ_CUDA(cudaMemcpy(pr->Wxg.ptr, g.Wxg.data(), g.Wxg.size() * sizeof(double), cudaMemcpyHostToDevice));
      HZ_CUDA(cudaMemcpy(pr->Wyg.ptr, g.Wyg.data(), g.Wyg.size() * sizeof(double), cudaMemcpyHostToDevice));
      HZ_CUDA(cudaMemcpy(pr->wxs.ptr, g.Wxs.data(), g.Wxs.size() * sizeof(double), cudaMemcpyHostToDevice));
      HZ_CUDA(cudaMemcpy(pr->wys.ptr, g.Wys.data(), g.Wys.size() * sizeof(double), cudaMemcpyHostToDevice));
      // source and boundary default to zero
      HZ_TRY(pr->f.ensure((size_t)g.n * 2 * sizeof(double)));
      HZ_CUDA(cudaMemset(pr->f.ptr, 0, (size_t)g.n * 2 * sizeof(double)));
      const size_t nbd = (size_t)(2 * g.NXg + 2 * g.NYg) * 2 * sizeof(double);
      HZ_TRY(pr->gb.ensure(nbd));
      HZ_CUDA(cudaMemset(pr->gb.ptr, 0, nbd));
      HZ_UPLOADS_DONE();
      HZ_CUDA(cudaStreamCreateWithFlags(&pr->stream, cudaStreamNonBlocking));
      return HZ_OK;
    }();
    if (s != HZ_OK) {
      delete pr;
      return s;
    }
    *out = pr;
    return HZ_OK;
  });
}

hz_status hz_problem_set(hz_problem pr, hz_field field, const double* data, int64_t count) {
  if (!pr) return fail(HZ_ERR_INVALID_ARG, "null problem");
  return guard([&]() { return set_field_host(*pr, field, data, count); });
}

hz_status hz_problem_set_device(hz_problem pr, hz_field field, const double* data, int64_t count, void* stream) {
  if (!pr || !data) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    const int64_t want = field_count(pr->g, field);
    if (want < 0 || count != want) return fail(HZ_ERR_INVALID_ARG, "wrong value count for field");
    const bool cplx_field = field == HZ_SOURCE || field == HZ_BOUNDARY;
    const int64_t nd = cplx_field ? 2 * count : count;
    // validate on the host (the check reads the data once; the copy stays device-side)
    std::vector<double> tmp((size_t)nd);
    HZ_TRY(use_device(*pr));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    HZ_CUDA(cudaMemcpyAsync(tmp.data(), data, nd * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaStreamSynchronize(st));
    if (field == HZ_OMEGA || field == HZ_WAVE_SPEED || field == HZ_TRANSMISSION || field == HZ_NODE_COORDS)
      return set_field_host(*pr, field, tmp.data(), count);
    if (!all_finite(tmp.data(), nd)) return fail(HZ_ERR_INVALID_ARG, "non-finite input");
    DevBuf& dst = field == HZ_SOURCE ? pr->f : pr->gb;
    HZ_TRY(dst.ensure(nd * sizeof(double)));
    HZ_CUDA(cudaMemcpyAsync(dst.ptr, data, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
    HZ_CUDA(cudaStreamSynchronize(st));
    pr->version++;
    return HZ_OK;
  });
}

void hz_problem_destroy(hz_problem pr) {
  if (!pr) return;
  cudaSetDevice(pr->device);
  for (cudaEvent_t e : pr->events) cudaEventDestroy(e);
  for (cudaEvent_t e : pr->gm_events) cudaEventDestroy(e);
  release_step_graphs(*pr);
  if (pr->pack_ready) cudaEventDestroy(pr->pack_ready);
  if (pr->join_event) cudaEventDestroy(pr->join_event);
  if (pr->stream) cudaStreamDestroy(pr->stream);
  delete pr;
}

hz_status hz_problem_nt(hz_problem pr, double cfl, int32_t* nt) {
  if (!pr || !nt) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(check_ready(*pr));
    if (!(cfl > 0.0)) return fail(HZ_ERR_INVALID_ARG, "cfl must be > 0");
    *nt = choose_nt(*pr, cfl);
    return HZ_OK;
  });
}

hz_status hz_solve(hz_problem pr, const hz_solve_opts* opts, double* u_out, hz_solve_report* report) {
  if (!pr || !u_out) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    hz_solve_opts o;
    opts_or_default(opts, &o);
    const size_t nb = (size_t)pr->g.n * 2 * sizeof(double);
    HZ_TRY(pr->uvec.ensure(nb));
    hz_status s = solve(*pr, o, pr->uvec.as<double>(), report, pr->stream);
    if (s != HZ_OK && s != HZ_ERR_NOT_CONVERGED) return s;
    HZ_CUDA(cudaMemcpyAsync(u_out, pr->uvec.ptr, nb, cudaMemcpyDeviceToHost, pr->stream));
    HZ_CUDA(cudaStreamSynchronize(pr->stream));
    return s;
  });
}

hz_status hz_solve_device(hz_problem pr, const hz_solve_opts* opts, double* u_out_dev, hz_solve_report* report,
                          void* stream) {
  if (!pr || !u_out_dev) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    hz_solve_opts o;
    opts_or_default(opts, &o);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (!is_default_stream(cs)) return solve(*pr, o, u_out_dev, report, cs);
    // A default stream cannot be captured into the step graphs: run on the
    // problem's own stream, ordered after the caller's work and before the
    // caller's later work.
    if (!pr->join_event) HZ_CUDA(cudaEventCreateWithFlags(&pr->join_event, cudaEventDisableTiming));
    HZ_CUDA(cudaEventRecord(pr->join_event, cs));
    HZ_CUDA(cudaStreamWaitEvent(pr->stream, pr->join_event, 0));
    const hz_status s = solve(*pr, o, u_out_dev, report, pr->stream);
    HZ_CUDA(cudaEventRecord(pr->join_event, pr->stream));
    HZ_CUDA(cudaStreamWaitEvent(cs, pr->join_event, 0));
    return s;
  });
}

hz_status hz_lambda_size(hz_problem pr, int64_t* n) {
  if (!pr || !n) return fail(HZ_ERR_INVALID_ARG, "null argument");
  *n = pr->g.lam_complex();
  return HZ_OK;
}

hz_status hz_prepare(hz_problem pr, int32_t nt, void* stream) {
  if (!pr) return fail(HZ_ERR_INVALID_ARG, "null problem");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return prepare(*pr, nt, static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_sweep(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol,
                   const double* lam_in, double* lam_out, const double* rhs_dev, double* u_sub, void* stream) {
  if (!pr || !lam_in || !lam_out) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (lam_in == lam_out) return fail(HZ_ERR_INVALID_ARG, "lam_in and lam_out must not alias");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return sweep(*pr, precision, nt, wh_iters, wh_tol, lam_in, lam_out, rhs_dev, u_sub,
                 static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_sweep_from(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol,
                        const double* lam_in, double* lam_out, const double* rhs_dev, const double* u0, double* u_sub,
                        void* stream) {
  if (!pr || !lam_in || !lam_out || !u0) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (lam_in == lam_out) return fail(HZ_ERR_INVALID_ARG, "lam_in and lam_out must not alias");
  if (precision == HZ_FP16_TRIAL || precision == HZ_BF16_TRIAL)
    return fail(HZ_ERR_UNSUPPORTED, "warm-started sweeps run in FP32 or FP64");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return sweep(*pr, precision, nt, wh_iters, wh_tol, lam_in, lam_out, rhs_dev, u_sub,
                 static_cast<cudaStream_t>(stream), u0);
  });
}

hz_status hz_sweep_rect(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol, int32_t sx0,
                        int32_t sy0, int32_t sw, int32_t sh, const double* lam_in, double* lam_out, const double* rhs_dev,
                        double* u_sub, void* stream) {
  if (!pr || !lam_in || !lam_out) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (lam_in == lam_out) return fail(HZ_ERR_INVALID_ARG, "lam_in and lam_out must not alias");
  const Geom& g = pr->g;
  if (sw < 1 || sh < 1 || sx0 < 0 || sy0 < 0 || sx0 + sw > g.Sx || sy0 + sh > g.Sy)
    return fail(HZ_ERR_INVALID_ARG, "subdomain rectangle outside the subdomain grid");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    const int rect[4] = {sx0, sy0, sw, sh};
    return sweep(*pr, precision, nt, wh_iters, wh_tol, lam_in, lam_out, rhs_dev, u_sub,
                 static_cast<cudaStream_t>(stream), nullptr, rect);
  });
}

hz_status hz_lambda_gather(hz_problem pr, const int32_t* slots, int32_t count, const double* lam, double* buf,
                           void* stream) {
  if (!pr || count < 0 || (count > 0 && (!slots || !lam || !buf))) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (count == 0) return HZ_OK;
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return launch_lambda_slots(slots, count, pr->g.NE, pr->g.L, lam, buf, /*gather=*/true,
                               static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_lambda_scatter(hz_problem pr, const int32_t* slots, int32_t count, const double* buf, double* lam,
                            void* stream) {
  if (!pr || count < 0 || (count > 0 && (!slots || !lam || !buf))) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (count == 0) return HZ_OK;
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return launch_lambda_slots(slots, count, pr->g.NE, pr->g.L, buf, lam, /*gather=*/false,
                               static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_sweep_packed(const hz_problem* problems, int32_t count, const int32_t* nts, int32_t wh_iters,
                          const double* const* lam_in, double* const* lam_out, const double* const* rhs,
                          double* const* u_sub, void* stream) {
  if (!problems || count < 0 || !nts || !lam_in || !lam_out) return fail(HZ_ERR_INVALID_ARG, "null argument");
  if (wh_iters < 0) return fail(HZ_ERR_INVALID_ARG, "wh_iters must be >= 0");
  if (count == 0) return HZ_OK;
  return guard([&]() -> hz_status {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    HZ_CUDA(cudaGetDevice(&dev));
    std::vector<WarpSweepArgs> descs(count);
    std::vector<int> offsets(count + 1, 0);
    for (int k = 0; k < count; ++k) {
      if (!problems[k] || !lam_in[k] || !lam_out[k]) return fail(HZ_ERR_INVALID_ARG, "null problem or buffer");
      if (lam_in[k] == lam_out[k]) return fail(HZ_ERR_INVALID_ARG, "lam_in and lam_out must not alias");
      Problem& pr = *problems[k];
      if (pr.device != dev) return fail(HZ_ERR_INVALID_ARG, "problem not on the current device");
      const Geom& g = pr.g;
      if (pr.mapped) return fail(HZ_ERR_UNSUPPORTED, "packed sweeps are built for Cartesian meshes only");
      const int shape = packed_shape_id(g.P, g.sny, g.nlx);
      if (shape < 0) return fail(HZ_ERR_UNSUPPORTED, "subdomain shape has no packed sweep variant");
      HZ_TRY(check_ready(pr));
      HZ_TRY(prepare(pr, nts[k], st));
      HZ_TRY(ensure_flags(pr));
      const double* rk = rhs ? rhs[k] : nullptr;
      double* uk = u_sub ? u_sub[k] : nullptr;
      descs[k].base = make_sweep_args(pr, true, nts[k], wh_iters, 0.0, lam_in[k], lam_out[k], rk, uk);
      descs[k].L = g.L;
      descs[k].shape = shape;
      warp_rows(g, &descs[k]);
      offsets[k + 1] = offsets[k] + g.L;
    }
    DevBuf dd, di;
    HZ_TRY(dd.ensure(descs.size() * sizeof(WarpSweepArgs)));
    HZ_TRY(di.ensure(offsets.size() * sizeof(int)));
    HZ_CUDA(cudaMemcpyAsync(dd.ptr, descs.data(), descs.size() * sizeof(WarpSweepArgs), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(di.ptr, offsets.data(), offsets.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    HZ_TRY(launch_sweep_packed(dd.as<WarpSweepArgs>(), di.as<int>(), count, st));
    HZ_CUDA(cudaStreamSynchronize(st));  // the tables are freed on return
    for (int k = 0; k < count; ++k) problems[k]->last_variant = kVariantPacked;
    return HZ_OK;
  });
}

hz_status hz_rhs(hz_problem pr, double* b, void* stream) {
  if (!pr || !b) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return rhs(*pr, b, static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_residual(hz_problem pr, const double* b, const double* u, double* r, double* norms2, void* stream) {
  if (!pr || !u || !r) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return residual(*pr, b, u, r, norms2, static_cast<cudaStream_t>(stream));
  });
}

hz_status hz_assemble_add(hz_problem pr, const double* u_sub, double* u, void* stream) {
  if (!pr || !u_sub || !u) return fail(HZ_ERR_INVALID_ARG, "null argument");
  return guard([&]() -> hz_status {
    HZ_TRY(use_device(*pr));
    return assemble_add(*pr, u_sub, u, static_cast<cudaStream_t>(stream));
  });
}

}  // extern "C"
