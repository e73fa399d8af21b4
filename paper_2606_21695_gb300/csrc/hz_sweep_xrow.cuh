// x part of the assembled stiffness apply for the register-resident sweeps
// (lane i owns node column i of a subdomain with at most 32 columns).
//
// (Kx p)_i / Wx_i with Kx the assembled 1D stiffness (Sec. 4: sum over the
// elements containing node i of the element matrix 2/hx Kref):
//   own element e = i / P (nodes eP .. eP+P, lane i is its node a = i % P):
//       sum_b Kref[a][b] p_{eP+b}
//   element e-1, only for a = 0 (lane i is that element's node P):
//       sum_b Kref[P][b] p_{(e-1)P+b}
// A lane gathers the P other nodes of its own element by indexed shuffles
// and contracts them with its row.  The element-(e-1) part of lane eP is
// formed by lane eP-1, which holds all of element e-1 after its own gather,
// and handed over by one more shuffle; its b = P term (lane eP's own value)
// stays in lane eP's centre coefficient.  P+1 shuffles per row instead of
// the 2P of a centred (2P+1)-tap stencil, for one extra FMA.
#pragma once

#include <cuda_runtime.h>

namespace hz {

template <int P>
struct XRow {
  int src[P + 1];    // src[k]: lane holding own-element node (a + k) mod (P+1), k = 1..P
  float kown[P + 1];  // kown[k]: coefficient of that node (k = 0: the lane itself)
  float kl[P + 1];    // kl[k]: element-(e-1) coefficient for the right neighbour (k = 1 unused)

  // Kref: (P+1)^2 reference stiffness (row a), kxs = 2/hx, wx(i) = lumped
  // 1D weight of column i; columns >= nlx are dead (all coefficients 0).
  template <typename WX>
  __device__ __forceinline__ void init(int lane, int nlx, int sxe, const double* Kref, double kxs, WX wx) {
    const int a = lane % P, e = lane / P;
    const bool live = lane < nlx;
    const bool own = live && e < sxe;
    const bool left = live && a == 0 && e >= 1;
    const double s_me = live ? kxs / wx(lane) : 0.0;
    // the right neighbour receives kl-part iff it is an element's first node
    // with an element to its left (a + 1 == P) and exists
    const bool sends = live && (a == P - 1) && (lane + 1 < nlx);
    const double s_nb = sends ? kxs / wx(lane + 1) : 0.0;
    for (int k = 0; k <= P; ++k) {
      const int b = (a + k) % (P + 1);
      src[k] = (e * P + b) & 31;
      double v = 0.0;
      if (own) v += Kref[a * (P + 1) + b];
      if (k == 0 && left) v += Kref[P * (P + 1) + P];  // lane is node P of element e-1
      kown[k] = (float)(v * s_me);
      // element e-1 of the neighbour is this lane's own element: row P
      kl[k] = (sends && k != 1) ? (float)(Kref[P * (P + 1) + b] * s_nb) : 0.f;
    }
  }

  // Returns (Kx p)_i / Wx_i for the row value pj of this lane.
  __device__ __forceinline__ float apply(float pj, int lane) const {
    float own = kown[0] * pj;
    float lp = kl[0] * pj;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const float v = __shfl_sync(0xffffffffu, pj, src[k]);
      own += kown[k] * v;
      if (k != 1) lp += kl[k] * v;
    }
    // lane 0 reads lane 31, whose part is 0 (dead, or the last column)
    return own + __shfl_sync(0xffffffffu, lp, (lane + 31) & 31);
  }
};

// The same x part for a band of 32 node columns c0 .. c0+31 of a wider
// subdomain (one warp of a cluster; the degree divides 32, so bands start on
// element boundaries).  Inside the band it is XRow's gather and hand-off;
// across the band's ends two halo inputs complete it: the node just past the
// band (needed by the band's last element: coefficient kR) and the P nodes
// before it (the element to the left of the band's first column: kL).
template <int P>
struct XRowBand {
  int src[P + 1];
  float kown[P + 1];
  float kl[P + 1];
  float kR;     // coefficient of column c0+32 (0 if this lane's element ends inside the band)
  float kL[P];  // coefficients of columns c0-P .. c0-1 (lane 0 of a band with c0 > 0 only)

  template <typename WX>
  __device__ __forceinline__ void init(int lane, int c0, int nlx, int sxe, const double* Kref, double kxs, WX wx) {
    const int c = c0 + lane;
    const int a = c % P, e = c / P;
    const bool live = c < nlx;
    const bool own = live && e < sxe;
    const bool left = live && a == 0 && e >= 1;
    const double s_me = live ? kxs / wx(c) : 0.0;
    // hand-off inside the band only (lane 31's part would belong to the next band)
    const bool sends = live && (a == P - 1) && (c + 1 < nlx) && (lane + 1 < 32);
    const double s_nb = sends ? kxs / wx(c + 1) : 0.0;
    kR = 0.f;
    for (int k = 0; k <= P; ++k) {
      const int b = (a + k) % (P + 1);
      const int sl = e * P + b - c0;  // lane of that node in this band (32: past its end)
      src[k] = sl & 31;
      double v = 0.0;
      if (own) v += Kref[a * (P + 1) + b];
      if (k == 0 && left) v += Kref[P * (P + 1) + P];
      float kv = (float)(v * s_me);
      if (k > 0 && sl >= 32) {
        kR = kv;
        kv = 0.f;
      }
      kown[k] = kv;
      kl[k] = (sends && k != 1) ? (float)(Kref[P * (P + 1) + b] * s_nb) : 0.f;
    }
    const bool lh = left && lane == 0;  // the element to the left lies in the previous band
    for (int b = 0; b < P; ++b) kL[b] = lh ? (float)(Kref[P * (P + 1) + b] * s_me) : 0.f;
  }

  // hR: p at column c0+32; hL[b]: p at column c0-P+b.
  __device__ __forceinline__ float apply(float pj, int lane, float hR, const float (&hL)[P]) const {
    float own = kown[0] * pj;
    float lp = kl[0] * pj;
#pragma unroll
    for (int k = 1; k <= P; ++k) {
      const float v = __shfl_sync(0xffffffffu, pj, src[k]);
      own += kown[k] * v;
      if (k != 1) lp += kl[k] * v;
    }
    own += kR * hR;
#pragma unroll
    for (int b = 0; b < P; ++b) own += kL[b] * hL[b];
    return own + __shfl_sync(0xffffffffu, lp, (lane + 31) & 31);  // lane 31 sends nothing
  }
};

// Edge-column correction of the p-dot update of a row.  The interior update
// is f = p-dot - beta' A p; the two edge lanes add (alpha - 1) p-dot +
// beta b_re cos + beta b_im sin + gamma p with (alpha - 1, beta b_re,
// beta b_im, gamma) read from shared memory (gamma = -beta x the interface
// boundary mass of a generalised transmission condition, 0 by default).
// Only the edge lanes load (no shared-memory traffic for interior lanes) and
// no per-row default values are needed.
template <bool RM = true>
__device__ __forceinline__ float edge_fix(float f, float pd, float p, const float4* row, bool edge, float c, float s) {
  if (edge) {
    const float4 e = *row;
    f += e.x * pd + e.y * c + e.z * s;
    if (RM) f += e.w * p;  // RM = false: the boundary mass is known to be zero
  }
  return f;
}

}  // namespace hz
