// Problem state behind the opaque hz_problem handle.
#pragma once

#include <string>
#include <vector>

#include "hz_internal.h"

namespace hz {

class Packer;

// Owning pinned host buffer (for the small device-to-host reads of the outer loop).
struct HostBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  HostBuf() = default;
  HostBuf(const HostBuf&) = delete;
  HostBuf& operator=(const HostBuf&) = delete;
  ~HostBuf();
  hz_status ensure(size_t nbytes);
  template <typename T>
  T* as() const { return static_cast<T*>(ptr); }
};

}  // namespace hz

struct hz_problem_s {
  hz::Geom g;
  int device = 0;
  cudaStream_t stream = nullptr;
  double omega = 0.0, cmax = 0.0, sigma = 0.0;
  double robin_eta = 0.0, robin_zeta = 1.0;  // interface condition d_n + k (eta - i zeta)
  bool has_c = false, has_omega = false;
  int version = 0;            // bumped on every field change
  int prepared_nt = 0, prepared_version = -1;
  long long sweeps_launched = 0;
  int last_variant = 0;       // sweep kernel used by the last sweep (kVariant*)
  int last_shape = 0;         // and its Choice::ty
  bool autotune = false;      // use / fill the tuned kernel choice for this shape
  hz::Packer* packer = nullptr;    // set while the solve's sweeps go out in packed launches
  cudaEvent_t pack_ready = nullptr;  // marks the stream position of a packed sweep request
  cudaEvent_t join_event = nullptr;  // orders a solve on the problem's stream with a caller's default stream
  // fields (global node grid)
  hz::DevBuf c, f, gb;
  // 1D weight tables
  hz::DevBuf Wxg, Wyg, wxs, wys;
  // leapfrog coefficients for prepared_nt
  hz::DevBuf beta64, alpha64, beta32, alpha32, kedge, tab64, tab32;
  // solver workspace
  hz::DevBuf bvec, rvec, uvec, usub, gv, xv, tv, V, part, small, flags, hcol;
  hz::DevBuf uwarm;  // subdomain solutions carried between sweeps (opts.wh_warm)
  hz::DevBuf Vg, Zg;  // global Krylov and preconditioned vectors of the FGMRES refinement
  hz::HostBuf hsmall, hcol_host;
  std::vector<cudaEvent_t> gm_events;  // one per Arnoldi step of a cycle
  // CUDA graphs of the Arnoldi step's vector work, one per step index of the
  // GMRES cycle, valid while step_graph_key (buffers, sizes) is unchanged
  std::vector<cudaGraphExec_t> step_graphs;
  std::vector<long long> step_graph_kernels;
  std::vector<const void*> step_graph_key;
  // general convex quadrilaterals (HZ_NODE_COORDS): geometry from node coordinates
  bool mapped = false;
  double mapped_mu = 0.0;      // element bound of lambda_max(W^-1 A), geometry only
  std::vector<double> mapped_D;  // (P+1)^2 differentiation matrix
  hz::DevBuf mgeo64, mgeo32, mWs, mEs, mshare;  // per subdomain
  hz::DevBuf mgeog, mWg, mHw, mbw, mflux;        // global (residual, right-hand side)
  // per-sweep CUDA events while a solve runs (report.sweep_seconds)
  bool time_sweeps = false;
  size_t ev_used = 0;
  std::vector<cudaEvent_t> events;
};

namespace hz {
using Problem = hz_problem_s;
constexpr int kVariantAuto = 0, kVariantBlock = 1, kVariantWarp = 2, kVariantCluster = 3, kVariantPacked = 4,
              kVariantClusterBand = 5, kVariantMapped = 6;
int sweep_variant();
struct Choice {
  int variant;  // kVariantBlock / kVariantWarp / kVariantCluster
  int ty;       // block kernel: rows per thread (0 = by size, 1 = P, 2 = 2P);
                // register-resident kernel: warps per subdomain (0/1, 2, 4)
};
std::string tune_key(const Geom& g, int precision);
bool lookup_choice(const std::string& key, Choice* out);
void store_choice(const std::string& key, Choice c);
hz_status autotune(Problem& pr, int precision, int nt, int m_wh, cudaStream_t st);
int choose_nt(const Problem& pr, double cfl);
hz_status prepare(Problem& pr, int nt, cudaStream_t st);
hz_status sweep(Problem& pr, int precision, int nt, int m_wh, double wh_tol, const double* lam_in, double* lam_out,
                const double* rhs, double* u_sub, cudaStream_t st,
                const double* u0 = nullptr, const int* rect = nullptr);
hz_status residual(Problem& pr, const double* b, const double* u, double* r, double* norms2_dev, cudaStream_t st);
hz_status rhs(Problem& pr, double* b, cudaStream_t st);
hz_status assemble_add(Problem& pr, const double* u_sub, double* u, cudaStream_t st);
hz_status solve(Problem& pr, const hz_solve_opts& o, double* u, hz_solve_report* rep, cudaStream_t st);
// The options a solve runs with: wh_iters = 0 together with a WaveHoltz
// tolerance stands for the default cap of kDefaultWhCap iterations.
constexpr int kDefaultWhCap = 1000;
hz_solve_opts effective_opts(const hz_solve_opts& o);
hz_status check_ready(const Problem& pr);
// Geometry of a mapped mesh from 2n node coordinates (x, y interleaved):
// validates J > 0 at every GLL node and uploads the metric and weights.
hz_status set_node_coords(Problem& pr, const double* xy);
void release_step_graphs(Problem& pr);
bool is_default_stream(cudaStream_t s);
unsigned long long launch_count();
void add_launches(long long n);
}  // namespace hz
