// Internal declarations shared by the host runtime (.cpp) and the kernels (.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hz.h"

namespace hz {

constexpr int kMaxP = 7;

// ------------------------------------------------------------- errors ----
void set_error(const std::string& msg);
hz_status fail(hz_status s, const std::string& msg);
hz_status cuda_fail(cudaError_t e, const char* what);
void note_launch();  // counts kernel launches (hz_kernel_launches)

#define HZ_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::hz::cuda_fail(e_, #call); \
  } while (0)

#define HZ_TRY(call)                     \
  do {                                   \
    hz_status s_ = (call);               \
    if (s_ != HZ_OK) return s_;          \
  } while (0)

// Host-to-device copies from pageable memory and memsets issued on the legacy
// default stream may return before the data are in device memory, and the
// problems' non-blocking streams are not ordered after that stream: every
// upload of problem data waits for the legacy stream before returning.
#define HZ_UPLOADS_DONE() HZ_CUDA(cudaStreamSynchronize(nullptr))

// ------------------------------------------------------- device memory ----
// Owning device buffer (cudaMalloc on the problem's device).
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  hz_status ensure(size_t nbytes);  // grows (contents not kept)
  void release();
  template <typename T>
  T* as() const { return static_cast<T*>(ptr); }
};

// --------------------------------------------------------- mesh geometry ----
struct Geom {
  double x0, x1, y0, y1, hx, hy;
  int nx, ny, P, snx, sny;
  int Sx, Sy, L;          // subdomain grid
  int NXg, NYg;           // global nodes per direction
  int nlx, nly, NE;       // subdomain nodes per direction, lambda slot length
  int64_t n;              // global nodes
  std::vector<double> xi, w;        // GLL nodes / weights on [-1, 1]
  std::vector<double> Kref;         // (P+1)^2: integral of l_a' l_b' over [-1,1], row a
  std::vector<double> Wxg, Wyg;     // global lumped 1D weights
  std::vector<double> Wxs, Wys;     // subdomain lumped 1D weights
  int64_t sub_nodes() const { return (int64_t)nlx * nly; }
  int64_t lam_complex() const { return (int64_t)L * 4 * NE; }
};

hz_status build_geom(double x0, double x1, double y0, double y1, int nx, int ny, int P, int snx, int sny, Geom* g);
double max_eig_1d(const Geom& g, int n_el, double h);  // largest eig of W^-1 K, 1D subdomain

// ------------------------------------------------------------- kernels ----
struct SweepArgs {
  int nlx, nly, NE, Sx, Sy, sxe, sye, NXg, NS, snxP, snyP;
  int ty_force;  // block kernel rows per thread: 0 = by size, 1 = P, 2 = 2P
  int round_mode;  // FP32 block kernel: 0 none, 1 round p and p-dot to FP16, 2 to BF16 (trials)
  int Nt, m_wh;
  double wh_tol, sigma, omega, cpi, spi, two_over_nt;
  double kxs, kys, hx2, hy2;  // 2/hx, 2/hy, hx/2, hy/2
  double eta, zeta;           // interface condition d_n + k (eta - i zeta)
  double Kref[(kMaxP + 1) * (kMaxP + 1)];
  float Kref32[(kMaxP + 1) * (kMaxP + 1)];
  double w[kMaxP + 1];
  const void* beta;   // [L][nly][nlx] Real
  const void* alpha;  // [L][nly][nlx] Real
  const void* tab;    // [Nt+1] x 4 Real: cos(2 pi nu/Nt), sin(2 pi nu/Nt), kappa_nu, kappa_{nu+1/2}/omega
  const double* kedge;  // [L][4][NE] omega / c at edge nodes
  const double* wxs;    // [nlx]
  const double* wys;    // [nly]
  const double* rhs;    // global complex or null
  const double* lam_in;
  double* lam_out;
  double* u_sub;        // [L][nly][nlx] complex or null
  int* wh_iter_max;
  unsigned long long* wh_iter_sum;  // sum over subdomains of WaveHoltz iterations
  int* flags;           // bit 0: non-finite value seen
  const double* u0;     // [L][nly][nlx] complex or null: WaveHoltz starts from it instead of zero
  // rank-local sweeps (hz_sweep_rect): with rect_w > 0 the launch covers the
  // rect_w x (count / rect_w) subdomains of the grid starting at subdomain
  // column rect_x0, row rect_y0; every array keeps the whole problem's layout
  int rect_x0, rect_y0, rect_w, rect_h;
};

// Subdomains one launch sweeps: the rectangle's, or all L.
inline int sweep_count(const SweepArgs& a, int L) { return a.rect_w > 0 ? a.rect_w * a.rect_h : L; }
// Subdomain swept by the k-th block (or cluster, or warp group) of a launch.
__host__ __device__ __forceinline__ int sweep_subdomain(const SweepArgs& a, int k) {
  return a.rect_w > 0 ? (a.rect_y0 + k / a.rect_w) * a.Sx + a.rect_x0 + k % a.rect_w : k;
}

// Parameters of the warp-per-subdomain FP32 sweep (subdomains <= 32 node
// columns).  The assembled y-stiffness rows divided by the row weight are
// compile-time tables (hz_gll_const.h) times sy = 4/hy^2.
constexpr int kWarpMaxRows = 33;
struct WarpSweepArgs {
  SweepArgs base;
  int L;
  int shape;                                   // packed launches: shape id (packed_shape_id)
  float sy;                                    // 4 / hy^2
  float wyr[kWarpMaxRows];                     // hy/2 * (w_a [own element] + w_P [element below])
};
// Register-resident sweep with h warps per subdomain (1, 2 or 4).  Returns
// HZ_ERR_UNSUPPORTED (without launching) when no variant for (P, sub_ny, h)
// was compiled or the subdomain has more than 32 node columns.
hz_status launch_sweep_warp(int P, int sy, int h, const WarpSweepArgs& a, cudaStream_t st);

// Packed sweep of several problems in one launch (register-resident body, one
// warp per subdomain).  descs: R per-problem parameter sets in device memory
// (shape ids in descs[d].shape); offsets: R+1 running subdomain counts in
// device memory (item it belongs to the d with offsets[d] <= it < offsets[d+1]).
// packed_shape_id returns -1 when (P, sub_ny, nlx) has no packed variant.
int packed_shape_id(int P, int sny, int nlx);
hz_status launch_sweep_packed(const WarpSweepArgs* descs, const int* offsets, int R, cudaStream_t st);

// FP32 sweep of one subdomain per thread-block cluster (column bands, halo
// exchange through distributed shared memory).  HZ_ERR_UNSUPPORTED when no
// cluster shape fits.
hz_status launch_sweep_cluster(int P, const SweepArgs& a, int L, cudaStream_t st);
// The same cluster sweep in FP64 (the plain-FP64 path for subdomains too
// large for one block).
hz_status launch_sweep_cluster_f64(int P, const SweepArgs& a, int L, cudaStream_t st);

// FP32 sweep of subdomains wider than 32 node columns by a cluster of CTAs,
// one per 32-column band, one warp per row band, state in registers (degree
// 1, 2 or 4; fixed WaveHoltz count or per-subdomain tolerance).  HZ_ERR_UNSUPPORTED when no compiled
// shape fits.
hz_status launch_sweep_cband(int P, const SweepArgs& a, int L, cudaStream_t st);

// Launches the sweep in Real = float (fp32 = true) or double.  Returns
// HZ_ERR_UNSUPPORTED when no compiled variant fits the subdomain.
hz_status launch_sweep_f32(int P, const SweepArgs& a, int L, cudaStream_t st);
hz_status launch_sweep_f64(int P, const SweepArgs& a, int L, cudaStream_t st);
inline hz_status launch_sweep(bool fp32, int P, const SweepArgs& a, int L, cudaStream_t st) {
  return fp32 ? launch_sweep_f32(P, a, L, st) : launch_sweep_f64(P, a, L, st);
}

struct PrepArgs {
  int nlx, nly, NE, Sx, Sy, NXg, snxP, snyP;
  double theta, sigma, omega;
  double zeta;          // interface damping factor (outer edges: 1)
  const double* c;      // global
  const double* wxs;
  const double* wys;
  // mapped meshes: per-node lumped weights [L][nly][nlx] and per-edge-node
  // arc-length weights [L][4][NE] replace the products of wxs, wys (null: Cartesian)
  const double* Wsub;
  const double* Esub;
  double* beta64;
  double* alpha64;
  float* beta32;
  float* alpha32;
  double* kedge;
};
hz_status launch_prepare(const PrepArgs& a, int L, cudaStream_t st);

struct GlobalArgs {
  int NXg, NYg, nx, ny, P;
  double omega, kxs, kys, hx2, hy2;
  double Kref[(kMaxP + 1) * (kMaxP + 1)];
  double w[kMaxP + 1];
  // assembled 1D stiffness rows by node class (class a = node a of an
  // element, 0 < a < P or a = 0 with elements on both sides; class P: first
  // node of the mesh; class P+1: last node), taps -P..P, scaled by 2/hx (Kx)
  // or 2/hy (Ky); built on the host
  double Kx[kMaxP + 2][2 * kMaxP + 1];
  double Ky[kMaxP + 2][2 * kMaxP + 1];
  const double* c;
  const double* Wxg;
  const double* Wyg;
};
// b = (f, phi) + <g, phi>; f: n complex; gb: boundary S,E,N,W complex.
hz_status launch_rhs(const GlobalArgs& a, const double* f, const double* gb, double* b, cudaStream_t st);
// r = b - K u (b may be null); partial sums of |r|^2, |b|^2 per block into part (2 per block);
// returns the number of blocks used through *nblocks.
hz_status launch_residual(const GlobalArgs& a, const double* b, const double* u, double* r, double* part,
                          int* nblocks, cudaStream_t st);
int residual_blocks(const GlobalArgs& a);
// out[k] = sum over blocks of part[blocks][k] for k < width, in fixed order.
hz_status launch_reduce_partials(const double* part, int nblocks, int width, double* out, cudaStream_t st);

struct AssembleArgs {
  int nlx, nly, Sx, Sy, NXg, NYg, snxP, snyP;
  const double* share;  // [L][nly][nlx] lumped-mass share of each copy; null: uniform mesh (1/count)
};
hz_status launch_assemble_add(const AssembleArgs& a, const double* u_sub, double* u, cudaStream_t st);

// ---- general convex quadrilaterals (isoparametric map from node coordinates)
// Element-local arrays are [.., ey, ex, b, a] (b along eta, a along xi) with
// (P+1)^2 nodes per element; metric entries are w_a w_b (G11, G12, G22).
struct MappedSweepArgs {
  SweepArgs base;        // coefficients, tables, lambda, rhs and outputs as for the Cartesian kernels
  const void* geo;       // [L][sny][snx][(P+1)^2][3] Real
  const double* wedge;   // [L][4][NE] arc-length GLL weights along the subdomain edges
  const double* share;   // [L][nly][nlx] lumped-mass share (splits a global right-hand side)
  int snx, sny;
  double D[(kMaxP + 1) * (kMaxP + 1)];  // D[q (P+1) + a] = l_a'(xi_q)
};
// HZ_ERR_UNSUPPORTED when the subdomain has more than 1024 nodes.
hz_status launch_sweep_mapped_f32(int P, const MappedSweepArgs& a, int L, cudaStream_t st);
hz_status launch_sweep_mapped_f64(int P, const MappedSweepArgs& a, int L, cudaStream_t st);
inline hz_status launch_sweep_mapped(bool fp32, int P, const MappedSweepArgs& a, int L, cudaStream_t st) {
  return fp32 ? launch_sweep_mapped_f32(P, a, L, st) : launch_sweep_mapped_f64(P, a, L, st);
}

struct MappedGlobalArgs {
  int NXg, NYg, nx, ny, P;
  double omega;
  double D[(kMaxP + 1) * (kMaxP + 1)];
  const double* c;
  const double* geo;     // [ny][nx][(P+1)^2][3] global element metric
  const double* W;       // [NYg][NXg] lumped weights
  const double* Hw;      // [NYg][NXg] outer-boundary arc-length weights (sum over the node's outer edges)
  const double* bw;      // [2 NXg + 2 NYg] outer edge weights in S, E, N, W order (as HZ_BOUNDARY)
  double* flux;          // [ny][nx][(P+1)^2][4] scratch (F1, F2 of Re u and Im u)
};
hz_status launch_rhs_mapped(const MappedGlobalArgs& a, const double* f, const double* gb, double* b, cudaStream_t st);
// r = b - K u as launch_residual (same partial-sum layout, 2 per block)
hz_status launch_residual_mapped(const MappedGlobalArgs& a, const double* b, const double* u, double* r, double* part,
                                 int* nblocks, cudaStream_t st);
int residual_mapped_blocks(const MappedGlobalArgs& a);

// ---- FP64 vector kernels for the outer Krylov iteration (complex, interleaved)
// part[blk][2k..2k+1] = partial sum over this block of conj(V_k) . w (complex) or
// real dot (real_dot = true, imaginary part 0), k = 0..nv-1; V_k = V + k*ld.
// With w_sub and w_out non-null the kernel dots x = w - w_sub instead and
// writes x to w_out (the Arnoldi vector (I - S) v from v and S v; w_out must
// not overlap V_0..V_{nv-1} or w).
int vec_blocks(int64_t n2);
// Streaming multiprocessors of the current device (looked up once per device).
int sm_count();
hz_status launch_multi_dot(const double* V, int64_t ld, int nv, const double* w, const double* w_sub, double* w_out,
                           int64_t n2, bool real_dot, double* part, int nblocks, cudaStream_t st);
// w -= sum_k h[k] V_k  (h complex on device, nv entries).  With norm_part
// non-null each block also writes the partial ||w_new||^2 to norm_part[2 blk]
// (0 to norm_part[2 blk + 1]) and *nblocks receives the block count.
int axpy_blocks(int64_t n2);
hz_status launch_multi_axpy(const double* V, int64_t ld, int nv, const double* h, double* w, int64_t n2,
                            bool real_coef, cudaStream_t st, double* norm_part = nullptr);
// y = x / sqrt(*norm2) with norm2 in device memory (0 if the norm is 0); y may
// be x.  With flags_src, also copies 4 status words to flags_dst.
hz_status launch_scale_inv_norm(const double* x, const double* norm2, double* y, int64_t n2, cudaStream_t st,
                                const int* flags_src = nullptr, int* flags_dst = nullptr);
// Transmission-data slots (l, e) listed in slots (2 int32 per slot, device):
// gather = true copies lam slot k (NE complex) to buf[k], else buf[k] to the
// lam slot; slots outside the L x 4 slots of lam are skipped (gather: zeros).
hz_status launch_lambda_slots(const int32_t* slots, int count, int NE, int L, const double* src, double* dst,
                              bool gather, cudaStream_t st);
// y = a*x + b*y
hz_status launch_axpby(double a, const double* x, double b, double* y, int64_t n2, cudaStream_t st);

}  // namespace hz

// Library-side objects behind the opaque handles.
struct hz_mesh_s {
  hz::Geom g;
};
