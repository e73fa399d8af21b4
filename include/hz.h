/*
 * hz -- GPU domain-decomposition Helmholtz solver (WaveHoltz subdomain solves).
 *
 * C ABI of the library libhz.so.  The method is that of "Efficient Domain
 * Decomposition for the Helmholtz Equation on GPUs" (arXiv 2606.21695):
 *   - problem: -Lap u - k^2 u = f in Omega, d_n u - i k u = g on dOmega,
 *     k = omega / c(x), time convention e^{-i omega t}      (Sec. 2, eq. (Helmholtz))
 *   - discretisation: degree-P GLL spectral elements on a structured quad
 *     mesh, lumped M and H: (A - i omega H - omega^2 M) u = b
 *                                                   (Sec. 4, eq. (discrete-helmholtz))
 *   - non-overlapping subdomains exchanging zeroth-order transmission data
 *     lambda, updated by lambda_{r,l} = -lambda_{l,r} - 2 i k u_l on the
 *     interface                                       (Sec. 3, eq. (lambda-iteration);
 *     the sign of the 2ik term is read as minus, which makes the DD fixed
 *     point equal to the global discrete solution)
 *   - each subdomain solved by WaveHoltz (Sec. 5, eq. (WaveHoltz), modified
 *     leapfrog), all subdomains in one launch per DD sweep (Sec. 6,
 *     Algorithm 1): one warp, a few warps, one block or one thread-block
 *     cluster per subdomain, by subdomain size
 *   - outer iteration: GMRES on the transmission data (Sec. 3, Krylov
 *     acceleration) inside FP64 refinement on the global residual, defect
 *     correction or flexible GMRES (Sec. 7: the DD cycle is a preconditioner
 *     and may run in lower precision).
 *
 * Conventions for every function below:
 *   - Return value: HZ_OK or an error code; hz_last_error() gives the message
 *     of the calling thread's last failure.  No function aborts the process.
 *   - Handles are owned by the library until the matching *_destroy.
 *   - Host arrays are owned by the caller and copied on entry / written on exit.
 *   - Complex arrays are interleaved (re, im) FP64.
 *   - Node arrays are on the global node grid of (nx*P+1) x (ny*P+1) nodes,
 *     x index fastest.
 *   - "device" pointers are CUDA device addresses on the problem's device;
 *     "stream" is a cudaStream_t (NULL = legacy default stream).  Device
 *     entry points enqueue work on that stream; they may synchronise it where
 *     noted.
 *   - Calls on one problem handle are not thread-safe; server calls are.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HZ_API __attribute__((visibility("default")))
#else
#define HZ_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hz_mesh_s* hz_mesh;
typedef struct hz_problem_s* hz_problem;
typedef struct hz_server_s* hz_server;

typedef enum {
  HZ_OK = 0,
  HZ_ERR_INVALID_ARG = 1, /* bad size, null pointer, non-finite or non-positive data */
  HZ_ERR_OOM = 2,         /* device or host allocation failed */
  HZ_ERR_CUDA = 3,        /* a CUDA call failed (message carries the CUDA error) */
  HZ_ERR_NOT_CONVERGED = 4, /* tolerance not met within max_sweeps / max_refine */
  HZ_ERR_DIVERGED = 5,    /* non-finite values (e.g. time step beyond the CFL limit) */
  HZ_ERR_TIMEOUT = 6,     /* a wait ran out (server poll) */
  HZ_ERR_BUSY = 7,        /* admission refused: HBM budget or queue full */
  HZ_ERR_NOT_FOUND = 8,   /* unknown ticket */
  HZ_ERR_INTERNAL = 9,
  HZ_ERR_UNSUPPORTED = 10 /* a size or degree outside the compiled kernels */
} hz_status;

/* Precision of the subdomain WaveHoltz loop (Sec. 7).  The outer GMRES,
 * refinement and global residual are always FP64.  The two trials keep the
 * wave state p, p-dot rounded to 16 bits after every update (arithmetic and
 * filter sums in FP32); they exist to report their error, not for speed. */
typedef enum { HZ_FP64 = 0, HZ_FP32_REFINE = 1, HZ_FP16_TRIAL = 2, HZ_BF16_TRIAL = 3 } hz_precision;

/* Outer iteration on the transmission data (Sec. 3).
 * GMRES: complex GMRES(m) on (I - S) lambda = g (S: homogeneous sweep).
 * PLAIN: the fixed-point iteration lambda <- S lambda + g of eq. (lambda-iteration).
 * RGMRES: real GMRES on the (re, im)-interleaved lambda vector; exact for a
 *         fixed WaveHoltz count, where the sweep is only real-linear. */
typedef enum { HZ_OUTER_GMRES = 0, HZ_OUTER_PLAIN = 1, HZ_OUTER_RGMRES = 2 } hz_outer;

/* FP64 refinement around the DD solves (Sec. 7: the DD cycle is a
 * preconditioner and may run in lower precision).
 * DEFECT: defect correction u <- u + DD(b - K u).
 * FGMRES: flexible GMRES on K u = b in FP64, right-preconditioned by the DD
 *         solve: each Krylov step is one DD solve (to inner_tol) and one K
 *         apply; the solution minimises the residual over all corrections of
 *         a cycle of refine_restart steps.  Converges where defect correction
 *         stagnates because the FP32 DD solve is accurate to only a fraction
 *         in a few ill-conditioned directions; costs two global vectors per
 *         step of the cycle. */
typedef enum { HZ_REFINE_DEFECT = 0, HZ_REFINE_FGMRES = 1 } hz_refine;

typedef enum {
  HZ_WAVE_SPEED = 0, /* n real values, finite and > 0 (c at every node) */
  HZ_OMEGA = 1,      /* 1 real value > 0 */
  HZ_SOURCE = 2,     /* n complex values (f at every node) */
  HZ_BOUNDARY = 3,   /* 2*(nx*P+1) + 2*(ny*P+1) complex values of g on the outer
                        edges in the order S, E, N, W, each along increasing x
                        (S, N) or y (E, W); corners carry one value per edge */
  HZ_TRANSMISSION = 4, /* 2 real values (eta >= 0, zeta > 0): the interface condition
                        B = d_n + k (eta - i zeta) used between subdomains (default
                        eta = 0, zeta = 1: B = d_n - i k, Sec. 3); eta > 0 adds a
                        boundary mass that damps evanescent interface modes (the
                        improved transmission conditions of Sec. 8).  The converged
                        solution does not depend on it, only the iteration count. */
  HZ_NODE_COORDS = 5  /* 2n real values: physical (x, y) of every global node, interleaved,
                         x-fastest in the mesh's logical node order.  Makes the mesh one of
                         general convex quadrilaterals (Sec. 4): each element is the
                         isoparametric degree-P image of the reference square through its
                         (P+1)^2 nodes; stiffness, lumped mass and boundary weights then
                         carry the map's metric.  The Jacobian must be positive at every
                         GLL node (else HZ_ERR_INVALID_ARG).  Subdomains must have at most
                         1024 nodes; FP64 and FP32-with-refinement solves only.  Without
                         it the mesh is the Cartesian grid of hz_mesh_create. */
} hz_field;

typedef struct {
  int32_t precision;     /* hz_precision */
  double tol;            /* stop when ||b - K u||_2 <= tol ||b||_2 (global, FP64) */
  int32_t max_sweeps;    /* budget of DD sweeps over the whole solve */
  int32_t outer;         /* hz_outer */
  int32_t gmres_restart; /* GMRES restart length m */
  int32_t wh_iters;      /* WaveHoltz iterations per sweep (maximum if wh_tol > 0; 0 with
                            wh_tol > 0: at most 1000) */
  double wh_tol;         /* > 0: a subdomain stops when ||u^{m+1}-u^m|| <= wh_tol ||u^{m+1}|| */
  int32_t nt_override;   /* > 0: time steps per period; 0: from the CFL rule */
  double cfl;            /* dt = cfl * 2 / (c_max sqrt(lx + ly)) */
  double inner_tol;      /* relative tolerance of each DD solve (GMRES on lambda) */
  int32_t max_refine;    /* maximum FP64 refinement steps */
  int32_t autotune;      /* 1: time the sweep kernel variants once per subdomain shape, use the fastest */
  int32_t wh_adaptive;   /* 1: per refinement step, WaveHoltz stops at tolerance clamp(0.1 * current
                            relative residual, wh_tol (or 1e-6), 1e-2), at most wh_iters iterations
                            (the variable inner tolerance of Sec. 5 / Sec. 8) */
  int32_t pack;          /* 1: in hz_solve_batch and the server, the sweeps of concurrent solves are
                            issued together, one packed launch per outer step covering every
                            subdomain of every member (FP32 sweeps with a fixed WaveHoltz count
                            on subdomains of at most 32 node columns and degree 1..5; other
                            solves run unpacked).  Ignored by hz_solve. */
  int32_t graphs;        /* 1: the vector work of each GMRES (Arnoldi) step -- Gram-Schmidt dots and
                            updates, norm, normalisation, read-back of the Hessenberg column -- is
                            captured once per step index as a CUDA graph and replayed in later
                            cycles (one launch instead of about ten per step) */
  int32_t gs_passes;     /* classical Gram-Schmidt passes per Arnoldi step (Sec. 3's Krylov
                            acceleration): 1 = one pass (half the FP64 work; orthogonality is lost
                            gradually over a restart cycle, which can cost iterations but not accuracy:
                            every DD solve is a correction that the FP64 refinement loop checks
                            against the true residual), 2 = one pass plus a full reorthogonalisation
                            (basis orthogonal to rounding).  Other values: HZ_ERR_INVALID_ARG. */
  int32_t wh_warm;       /* 1: each sweep of the plain fixed-point iteration (outer = HZ_OUTER_PLAIN)
                            starts WaveHoltz from the previous sweep's subdomain solutions instead of
                            zero (Sec. 8: subdomain solves loose at first, tighter as lambda settles;
                            with wh_tol > 0 the WaveHoltz iteration count falls as the outer iteration
                            converges).  The sweep then depends on the previous iterate, so the GMRES
                            outer iterations refuse it (HZ_ERR_INVALID_ARG).  Default 0. */
  int32_t refine;        /* hz_refine: the FP64 refinement (default HZ_REFINE_DEFECT); with FGMRES,
                            max_refine bounds the DD solves (preconditioner applications) */
  int32_t refine_restart; /* FGMRES cycle length, 1..200 (default 30) */
} hz_solve_opts;

typedef struct {
  int32_t sweeps;        /* DD sweeps (kernel launches of the subdomain solve) */
  int32_t refinements;   /* FP64 refinement steps: defect corrections, or the DD solves applied
                            as preconditioner by the FGMRES refinement */
  int32_t nt;            /* time steps per period used */
  int32_t wh_iters_max;  /* largest WaveHoltz iteration count of any subdomain */
  double rel_residual;   /* final ||b - K u|| / ||b|| (FP64, global) */
  double seconds;        /* wall time of the solve */
  int64_t dof_updates;   /* sum over sweeps of subdomain nodes x (N_t - 1) x WaveHoltz iterations */
  int32_t gmres_iters;   /* total GMRES iterations */
  int32_t sweep_variant; /* kernel of the last sweep: 1 block, 2 warp per subdomain, 3 cluster,
                            4 packed with other solves, 5 cluster of warp bands, 6 mapped mesh */
  int32_t sweep_shape;   /* its configuration: warps per subdomain (2), rows per thread in units
                            of the degree (1, 3; 0 = chosen by size) */
  double sweep_seconds;  /* device time of the sweep kernels (CUDA events on the solve's stream) */
} hz_solve_report;

/* Defaults: FP64, tol 1e-8, 2000 sweeps, GMRES(60), 20 WaveHoltz iterations,
 * no wh_tol, CFL 0.9, inner_tol 1e-2, 20 refinements, autotune, pack and
 * graphs on, one Gram-Schmidt pass, no warm start, defect-correction
 * refinement (FGMRES cycle 30 when selected). */
HZ_API void hz_default_opts(hz_solve_opts* opts);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to n bytes).  Returns HZ_OK. */
HZ_API hz_status hz_last_error(char* buf, size_t n);

/* Number of CUDA kernels this library has launched in the process so far
 * (all devices, all threads).  Not part of the method; for accounting. */
HZ_API hz_status hz_kernel_launches(uint64_t* count);

/* Measured FMA-pipe rate of the current device (a measurement utility; the
 * paper has no counterpart).  Runs a kernel of independent fused
 * multiply-adds only -- FP32 for precision HZ_FP32_REFINE, FP64 for HZ_FP64 --
 * on 4 blocks of 256 threads per SM, each thread iters x 128 FMAs, timed with
 * CUDA events on a private stream after one shorter warm-up launch.  Writes
 * the achieved TFLOP/s (2 flops per FMA) and the timed launch's milliseconds.
 * This is the denominator the sweep kernels' roofline fractions are quoted
 * against.  Errors: HZ_ERR_INVALID_ARG for another precision, iters < 1 or a
 * null pointer; HZ_ERR_CUDA if the launch fails. */
HZ_API hz_status hz_fma_peak(int32_t precision, int32_t iters, double* tflops, double* ms);

/* ------------------------------------------------------------------ mesh --
 * Structured mesh of [x0,x1] x [y0,y1] with nx x ny quad elements of degree
 * P (1..7), split into subdomains of sub_nx x sub_ny elements (Sec. 3, Fig. 1;
 * Sec. 4).  sub_nx must divide nx and sub_ny divide ny.  Errors:
 * HZ_ERR_INVALID_ARG on bad sizes or an empty box. */
HZ_API hz_status hz_mesh_create(double x0, double x1, double y0, double y1, int32_t nx, int32_t ny, int32_t degree,
                         int32_t sub_nx, int32_t sub_ny, hz_mesh* out);
/* n = (nx*P+1)*(ny*P+1). */
HZ_API hz_status hz_mesh_num_nodes(hz_mesh mesh, int64_t* n);
/* Writes the 2n node coordinates (x, y) interleaved, x index fastest, into the
 * caller's buffer xy (GLL node positions, Sec. 4). */
HZ_API hz_status hz_mesh_node_coords(hz_mesh mesh, double* xy);
HZ_API void hz_mesh_destroy(hz_mesh mesh);

/* --------------------------------------------------------------- problem --
 * A problem on a mesh, resident on CUDA device `device`.  The problem keeps a
 * reference to the mesh (the mesh may be destroyed by the caller afterwards). */
HZ_API hz_status hz_problem_create(hz_mesh mesh, int32_t device, hz_problem* out);
/* Copies a field from host memory (count values as described by hz_field;
 * complex fields count complex numbers).  Validates finiteness and c > 0. */
HZ_API hz_status hz_problem_set(hz_problem pr, hz_field field, const double* data, int64_t count);
/* Same from device memory (copied device-to-device on `stream`, which is
 * synchronised). */
HZ_API hz_status hz_problem_set_device(hz_problem pr, hz_field field, const double* data, int64_t count, void* stream);
HZ_API void hz_problem_destroy(hz_problem pr);

/* Time steps per period from the CFL rule: N_t = max(3, ceil((2 pi/omega)/dt))
 * with dt = cfl * 2 / (c_max sqrt(lx + ly)), lx, ly the largest eigenvalues
 * of the 1D subdomain stiffness over its lumped mass (Sec. 5; the paper's
 * dt <= 2h/(p^2 c_max) is replaced by this exact bound). */
HZ_API hz_status hz_problem_nt(hz_problem pr, double cfl, int32_t* nt);

/* ------------------------------------------------------------------ solve --
 * Full solve to opts->tol: FP64 refinement on the global residual (Sec. 7),
 * either defect correction u <- u + DD(b - K u) or flexible GMRES on K u = b
 * with the DD solve as right preconditioner (opts->refine); each DD solve is
 * an outer iteration on lambda whose matvec is one sweep (one kernel launch
 * over all subdomains).  u_out: host buffer of n complex values.
 * Returns HZ_ERR_NOT_CONVERGED (report filled, u_out written) if the budget
 * runs out; HZ_ERR_DIVERGED (report filled) on non-finite values, a Krylov
 * operator norm beyond 1e8, or a refinement step or FGMRES cycle that
 * multiplied the residual by 1e4 or more. */
HZ_API hz_status hz_solve(hz_problem pr, const hz_solve_opts* opts, double* u_out, hz_solve_report* report);
/* (With the environment variable HZ_SOLVE_LOG set, hz_solve and hz_solve_device print the
 * residual after every refinement step, or the FGMRES residual estimate after every DD
 * solve, to stderr: progress of long solves.) */
/* Same with the solution written to device memory u_out_dev (n complex),
 * ordered on `stream` (a default stream -- legacy or per-thread -- is joined
 * by events and the work runs on the problem's own stream). */
HZ_API hz_status hz_solve_device(hz_problem pr, const hz_solve_opts* opts, double* u_out_dev, hz_solve_report* report,
                          void* stream);

/* Solves count independent problems concurrently on their devices (batched
 * execution, continuous across sizes, degrees and frequencies): at most
 * max_concurrent solves (<= 0: all of them, up to 64) run at once, started in
 * decreasing order of estimated cost; with opts->autotune the sweep kernel of
 * each distinct subdomain shape is timed once first; with opts->pack the
 * sweeps of the running solves go out as one packed launch per outer step.  u_out[k] (host, n_k complex) may be
 * NULL; reports may be NULL; statuses[k] receives each solve's status.
 * Returns HZ_OK, HZ_ERR_NOT_CONVERGED if any solve ran out of budget, or the
 * first hard error (hz_last_error names the problem). */
HZ_API hz_status hz_solve_batch(const hz_problem* problems, int32_t count, const hz_solve_opts* opts,
                                int32_t max_concurrent, double* const* u_out, hz_solve_report* reports,
                                hz_status* statuses);

/* ------------------------------------------------- hot-path step calls --
 * These expose the individual steps of the path on device buffers.
 *
 * Transmission data layout ("lambda vector"): L*4*NE complex values,
 * L = number of subdomains (x index fastest), 4 edges per subdomain in the
 * order W, E, S, N, NE = max(sub_nx, sub_ny)*P + 1 nodes per edge along
 * increasing x (S, N) or y (W, E); unused tail entries and the slots of
 * edges on the outer boundary are zero on output. */
HZ_API hz_status hz_lambda_size(hz_problem pr, int64_t* n_complex);

/* Prepares the per-subdomain leapfrog coefficients (alpha, beta of Sec. 5)
 * for nt time steps per period.  Called implicitly by the functions below
 * when nt changes. */
HZ_API hz_status hz_prepare(hz_problem pr, int32_t nt, void* stream);

/* One DD sweep (Algorithm 1 on every subdomain, one thread block each, one
 * launch): assemble b from the split global source rhs (NULL = homogeneous)
 * and lam_in, run wh_iters WaveHoltz iterations (wh_tol as in
 * hz_solve_opts), write lam_out (lambda vector) and, if u_sub is not NULL,
 * the subdomain solutions (L x nly x nlx complex, nly = sub_ny*P+1,
 * nlx = sub_nx*P+1, subdomain-major).  precision: hz_precision of the loop. */
HZ_API hz_status hz_sweep(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol,
                   const double* lam_in, double* lam_out, const double* rhs, double* u_sub, void* stream);

/* hz_sweep with WaveHoltz started from u0 instead of zero (the warm start of
 * opts.wh_warm, Sec. 8): u0 holds subdomain solutions in the u_sub layout
 * (device, complex, L x nly x nlx), typically the previous sweep's; u0 may be
 * the same buffer as u_sub (each subdomain reads its start before it writes
 * its result).  Runs on the register-resident kernels (1, 2 or 4 warps per
 * subdomain: the autotuned shape) where they fit (FP32), else the block
 * kernel, or the mapped-mesh kernel.  16-bit trial precisions:
 * HZ_ERR_UNSUPPORTED. */
HZ_API hz_status hz_sweep_from(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol,
                               const double* lam_in, double* lam_out, const double* rhs, const double* u0,
                               double* u_sub, void* stream);

/* Rank-local sweep for a problem split over several GPUs (Sec. 8: the DD
 * sweep partitions by subdomains and only interface data crosses between
 * GPUs).  Sweeps only the subdomains of the rectangle of subdomain columns
 * sx0 .. sx0+sw-1 and rows sy0 .. sy0+sh-1 (subdomain l = sy * S_x + sx),
 * with the arithmetic of hz_sweep, one launch.  lam_in, lam_out, rhs and
 * u_sub keep the whole problem's layouts (as hz_sweep).  Writes in lam_out:
 * the slots the rectangle's subdomains send to every neighbour -- inside the
 * rectangle, and the slots of neighbouring subdomains outside it (the cut
 * interfaces, to be sent to their owner: hz_lambda_gather) -- and zero in
 * its own outer-boundary slots; slots of its own subdomains that face
 * subdomains outside the rectangle are not written (their owner's sweep
 * produces them: hz_lambda_scatter).  u_sub (or NULL): solutions of the
 * rectangle's subdomains only.  Over a partition of the subdomain grid into
 * rectangles, the union of the rank-local sweeps plus the exchange gives
 * bitwise the lambda of one hz_sweep.  HZ_ERR_INVALID_ARG for a rectangle
 * outside the grid. */
HZ_API hz_status hz_sweep_rect(hz_problem pr, int32_t precision, int32_t nt, int32_t wh_iters, double wh_tol,
                               int32_t sx0, int32_t sy0, int32_t sw, int32_t sh, const double* lam_in,
                               double* lam_out, const double* rhs, double* u_sub, void* stream);

/* Packing of cut-interface transmission data for the exchange between GPUs
 * (Sec. 8).  slots: device array of count pairs (l, e) (int32: subdomain,
 * edge 0..3 = W, E, S, N) of a lambda vector; buf: device array of count x NE
 * complex values, slot k at buf[k NE .. (k+1) NE - 1].  gather copies the
 * slots of lam into buf (the send buffer); scatter copies buf into the slots
 * of lam (after the receive).  The slot lists of a sender and its receiver
 * must enumerate the same interfaces in the same order.  A slot outside the
 * lambda vector (l not in 0..L-1 or e not in 0..3) is skipped: gather writes
 * zeros for it, scatter writes nothing. */
HZ_API hz_status hz_lambda_gather(hz_problem pr, const int32_t* slots, int32_t count, const double* lam, double* buf,
                                  void* stream);
HZ_API hz_status hz_lambda_scatter(hz_problem pr, const int32_t* slots, int32_t count, const double* buf, double* lam,
                                   void* stream);

/* The same sweep for count problems in one packed launch (the batched form
 * used by hz_solve_batch and the server; Algorithm 1, Sec. 6): every
 * subdomain of every problem is swept by one warp, FP32, with nts[k] time
 * steps per period for problem k and a fixed wh_iters WaveHoltz iterations.
 * lam_in[k], lam_out[k], rhs[k] (or NULL), u_sub[k] (or NULL): device
 * buffers of problem k as in hz_sweep.  All problems must live on the
 * current device.  Returns after the launch has completed on `stream`.
 * HZ_ERR_UNSUPPORTED (nothing launched) if a problem's subdomain has more
 * than 32 node columns or a (degree, sub_ny) outside the packed variants
 * (degree 1 with sub_ny 4, 8, 16; degree 2 with 4, 8; degree 3 with 4, 8;
 * degrees 4, 5 with 4). */
HZ_API hz_status hz_sweep_packed(const hz_problem* problems, int32_t count, const int32_t* nts, int32_t wh_iters,
                                 const double* const* lam_in, double* const* lam_out, const double* const* rhs,
                                 double* const* u_sub, void* stream);

/* Global weak-form right-hand side b = (f, phi) + <g, phi> (Sec. 4), n complex. */
HZ_API hz_status hz_rhs(hz_problem pr, double* b, void* stream);

/* r = b - (A - i omega H - omega^2 M) u on the whole mesh, FP64, n complex
 * (Sec. 4, matrix-free).  If norms2 is not NULL it receives ||r||^2 and
 * ||b||^2 (2 doubles, device memory).  b may be NULL (treated as zero, so
 * r = -K u).  Uses library-owned scratch for the reduction. */
HZ_API hz_status hz_residual(hz_problem pr, const double* b, const double* u, double* r, double* norms2, void* stream);

/* Same as hz_residual, for callers that cannot allocate device memory (code
 * running inside someone else's CUDA graph capture, hosts whose allocator
 * belongs to another runtime, real-time loops that must not synchronise):
 * this entry point allocates nothing.  (The paper has no counterpart; it is
 * an interface convenience.)  The caller owns every array: c (n real wave
 * speeds), b (n complex, may be NULL = zero), u (n complex), r (n complex,
 * output), norms2 (2 doubles: ||r||^2, ||b||^2), all device memory on the
 * current device; mesh is the host-side mesh description.  Block partial
 * sums live in a fixed array in the library's device memory (2 MiB, held by
 * every device that loads the library until the process exits), which limits
 * the mesh to 2^17 blocks of 32 x 8 nodes (about 33.5 M nodes) and at most
 * 524280 node rows (65535 blocks of 8 rows); larger meshes return
 * HZ_ERR_UNSUPPORTED before anything is launched.  The first call on a
 * device looks up that array's device address (set-up): make it before any
 * stream capture.  All calls share the array, so calls that overlap on the
 * GPU race; serialise them on one stream.  The mesh is the Cartesian grid of
 * hz_mesh_create (node coordinates set on a problem with HZ_NODE_COORDS are
 * not seen here; use hz_residual on that problem). */
HZ_API hz_status hz_residual_noalloc(hz_mesh mesh, double omega, const double* c, const double* b, const double* u,
                                     double* r, double* norms2, void* stream);

/* u += mass-weighted average of the subdomain copies u_sub (the inverse of the
 * splitting of a global right-hand side by lumped-mass share). */
HZ_API hz_status hz_assemble_add(hz_problem pr, const double* u_sub, double* u, void* stream);

/* ------------------------------------------------------------------ server --
 * Continuous-batching request server on one device: submitted solves are
 * admitted against an HBM budget and advanced together, one sweep of every
 * active solve per scheduling tick. */
HZ_API hz_status hz_server_create(int32_t device, uint64_t hbm_budget_bytes, hz_server* out);
/* Snapshots the problem (fields are copied) and queues a solve. */
HZ_API hz_status hz_server_submit(hz_server srv, hz_problem pr, const hz_solve_opts* opts, uint64_t* ticket);
/* timeout_ms < 0 waits without limit, 0 polls.  On completion writes u_out
 * (host, n complex; may be NULL) and the report, sets *done = 1 and forgets
 * the ticket; otherwise *done = 0 and HZ_ERR_TIMEOUT after a positive
 * timeout.  The solve's own status is returned when done. */
HZ_API hz_status hz_server_poll(hz_server srv, uint64_t ticket, int32_t timeout_ms, double* u_out, hz_solve_report* report,
                         int32_t* done);
/* Latency percentiles (submit to completion) over completed requests,
 * completed solves per second since creation, device bytes held now. */
HZ_API hz_status hz_server_stats(hz_server srv, double* p50_ms, double* p99_ms, double* solves_per_s, uint64_t* hbm_in_use);
/* Cancels queued requests, finishes or abandons in-flight ones, frees all. */
HZ_API void hz_server_destroy(hz_server srv);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
