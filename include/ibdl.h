/*
 * ibdl.h -- C ABI of the GB300 (sm_103a) Immersed Boundary Double Layer
 * (IBDL) library.
 *
 * The library solves the Helmholtz boundary value problems of Leathers & Guy,
 * "Immersed Boundary Double Layer method" (arXiv:2203.12126):
 *
 *   Dirichlet (Sec. 2, eq. (pde)):           Delta u - k^2 u = g in Omega,
 *                                             u = U_b on Gamma,
 *   Neumann   (Sec. 4.4, eq. (pde neumann)):  Delta u - k^2 u = g in Omega,
 *                                             du/dn = V_b on Gamma,
 *
 * by embedding Omega in a periodic box C = [origin, origin + L)^d (d = 2, 3)
 * with n grid nodes per axis at origin + j h, h = L / n (Sec. 5.1), and
 * solving the well-conditioned second-kind boundary system of Sec. 5.3 /
 * Sec. 4.4 with unpreconditioned GMRES.  This library writes the operator as
 * L' = I - kappa Delta_h with kappa = 1 / k^2, so the paper's
 * L = Delta_h - k^2 = -(1/kappa) L'.  The boundary operators are then
 *
 *   A_D Q = Q/2 + kappa S* L'^{-1} S~ Q      (eq. (ibdl schur again))
 *   A_N U = kappa S* L'^{-1} S~ U - U/2      (eq. (Neumann saddle point))
 *
 * where S is the spread (Sec. 5.2, eq. (spread operator again2)), S* the
 * interpolation (eq. (interpolation again)), S~ Q = div_h(S (Q n)) (eq.
 * (Stilde)) with centred differences, Delta_h the 5-point (2D) or 7-point
 * (3D) Laplacian and delta_h the Peskin 4-point (eq. (delta eqn 2)) or the
 * cosine 4-point kernel.
 *
 * Conventions for every entry point:
 *   - Pointers to per-point arrays (length m) and grid arrays (n^d values,
 *     x fastest, then y, then z) may be DEVICE or HOST memory; the library
 *     tells them apart with cudaPointerGetAttributes.  Host arrays are
 *     copied to/from library-owned device staging buffers on the call's
 *     stream (pinned host memory makes those copies asynchronous).
 *   - The caller owns every pointer it passes; it must stay valid until the
 *     stream has finished the call.  The geometry handle owns its device
 *     workspaces until ibdl_destroy_geometry.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work asynchronously unless stated otherwise.
 *   - A handle is not thread-safe: one host thread (and one stream at a
 *     time) per handle.  Distinct handles are independent.
 *   - Errors: every function returns an ibdl_status; on failure nothing is
 *     written to the outputs unless stated otherwise, and
 *     ibdl_last_error_message() returns a description (per host thread).
 */
#ifndef IBDL_H_
#define IBDL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBDL_VERSION_MAJOR 0
#define IBDL_VERSION_MINOR 1

typedef enum {
  IBDL_OK = 0,
  IBDL_ERR_INVALID_ARG = 1,   /* bad size, pointer, kappa, bc, ... */
  IBDL_ERR_OOM = 2,           /* device allocation failed */
  IBDL_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  IBDL_ERR_NOT_CONVERGED = 4, /* GMRES hit max_iters; best iterate returned */
  IBDL_ERR_BREAKDOWN = 5,     /* Arnoldi produced a zero or non-finite norm */
  IBDL_ERR_NONFINITE = 6,     /* NaN/Inf in inputs or in the residual */
  IBDL_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
  IBDL_ERR_UNSUPPORTED = 8    /* valid request the library does not support */
} ibdl_status;

typedef enum { IBDL_DIRICHLET = 0, IBDL_NEUMANN = 1 } ibdl_bc;

/* Peskin's 4-point kernel, Sec. 5.2 eq. (delta eqn 2); or the cosine
 * 4-point kernel phi(r) = (1 + cos(pi r / 2)) / 4 on |r| < 2. */
typedef enum { IBDL_DELTA_PESKIN4 = 0, IBDL_DELTA_COS4 = 1 } ibdl_delta;

/* IBDL_FP64: every step in float64.
 * IBDL_FP32_REFINED: spread, FFT solve and interpolation in float32 inside
 * the GMRES iterations; Arnoldi, Givens and an outer residual-refinement loop
 * in float64.  The loop's residual b - A x and the right-hand side use the
 * IBDL_FP64_DF operator (finite-difference, non-completed geometries; the
 * others use the float64 operator).
 * IBDL_FP64_DF (ibdl_apply_precision only): float64 spread and
 * interpolation, FFT solve in double-float arithmetic (pairs of floats,
 * about 48 significant bits, float exponent range).  Agrees with the float64
 * operator to about 1e-14 relative, at a fraction of its cost on GPUs whose
 * float64 rate is low. */
typedef enum { IBDL_FP64 = 0, IBDL_FP32_REFINED = 1, IBDL_FP64_DF = 2 } ibdl_precision;

/* Discretisation of the PDE operator (Sec. 5.1, Sec. 6.2.1).  The divergence
 * inside S~ follows it (Sec. 5.2).
 * IBDL_DISC_FD: the 5/7-point Laplacian and centred differences.
 * IBDL_DISC_SPECTRAL: the Fourier-spectral Laplacian, symbol
 *   sum_c (2 pi k_c / L)^2, and spectral derivatives i 2 pi k_c / L, zero at
 *   the Nyquist mode.  Solves use the launch-based engine.  Batched solves,
 *   the server, ibdl_spread_div and ibdl_helmholtz (finite-difference
 *   operators) and the completed system return IBDL_ERR_UNSUPPORTED. */
typedef enum { IBDL_DISC_FD = 0, IBDL_DISC_SPECTRAL = 1 } ibdl_disc;

typedef struct ibdl_geometry_s* ibdl_geometry; /* opaque, library-owned */

/* Geometry of one IBDL problem (Sec. 5.1-5.2).  Copied at creation. */
typedef struct {
  int32_t dim;          /* 2 or 3 */
  int32_t n;            /* grid nodes per axis: a power of two, 16..2048 in 2D,
                           16..512 in 3D (larger grids need more shared memory
                           per float64 FFT item than a block can have) */
  double box_len;       /* L > 0; h = L / n */
  double origin[3];     /* lower box corner; nodes at origin + j h */
  int64_t m;            /* number of boundary points, 1..16776960 */
  const double* x;      /* point coordinates X_i, length m each; z only for */
  const double* y;      /* dim == 3 (may be NULL in 2D)                      */
  const double* z;
  const double* nx;     /* unit normals n_i pointing OUT of Omega (Sec. 4.1) */
  const double* ny;
  const double* nz;
  const double* w;      /* quadrature weights Delta s_i (arclength, Sec. 5.2)
                           or dA_i (area, Sec. 6.7) */
  double kappa;         /* > 0: L' = I - kappa Delta_h, k^2 = 1/kappa.
                           +INFINITY selects the Poisson equation (k = 0,
                           Sec. 5.4): kappa L'^{-1} becomes -Delta_0^{-1}, the
                           inverse of Delta_h returning the mean-zero field
                           (the k = 0 mode of every source is dropped, so a
                           forcing g~ must satisfy the solvability condition
                           of App. C, e.g. through the choice of g_e).
                           Dirichlet only. */
  int32_t delta;        /* ibdl_delta */
  int32_t bc;           /* ibdl_bc: selects A_D or A_N */
  int32_t precision;    /* ibdl_precision */
  int32_t disc;         /* ibdl_disc (0: finite difference) */
  double eta;           /* completed IBDL (Sec. 5.4 eq. (ibdl completed),
                           App. C): weight of the single layer eta S Q added
                           to S~ Q.  0 = the plain method.  eta > 0 needs
                           kappa = +INFINITY.  The unknown is then
                           z = (Q, u_bar), length m + 1 (z[m] = u_bar, the
                           field's mean), and the system is
                             Q/2 - S* Delta_0^{-1} (S~ + eta S) Q + u_bar
                                 = U_b - S* Delta_0^{-1} g~
                             eta sum_i w_i Q_i = h^d sum_j g~_j.
                           ibdl_apply, ibdl_solve (q_out, x0) and
                           ibdl_evaluate (q) then take length m + 1 vectors;
                           such geometries solve on the launch-based engine
                           and are not accepted by ibdl_solve_batched or the
                           server. */
} ibdl_geometry_desc;

typedef struct {
  double tol;           /* stop when ||b - A x||_2 / ||b||_2 <= tol (the
                           relative residual of Sec. 5.3); default 1e-8 */
  int32_t restart;      /* GMRES(restart), 1..64; default 30 */
  int32_t max_iters;    /* total inner iterations; default 500 */
  int32_t max_refine;   /* outer refinement steps (FP32_REFINED); default 8 */
  int32_t engine;       /* 0 (default): the whole solve in one persistent
                           cooperative kernel launch, no host round trip per
                           iteration; 1: host-driven loop of per-pass kernels
                           with a residual read-back per iteration */
  double inner_tol;     /* FP32_REFINED: relative tolerance of each inner
                           solve; default 1e-5 */
  const double* x0;     /* optional initial guess (length m), or NULL */
} ibdl_solve_opts;

typedef struct {
  int32_t iters;             /* total GMRES inner iterations (all cycles) */
  int32_t refine_steps;      /* outer refinement steps taken (0 for FP64) */
  int32_t matvecs;           /* operator applications, all precisions */
  int32_t n_history;         /* entries used in residual_history */
  double rel_residual;       /* final ||b - A x|| / ||b||: from a float64-grade
                                residual, or (FP32_REFINED) from a residual
                                updated after a small correction d as
                                r - A32 d, within 1e-5 ||d|| of the true
                                one, a bound the stopping test adds to it */
  double residual_history[256]; /* relative residual after each iteration */
  int32_t residual_updates;  /* FP32_REFINED: residuals updated by a float32
                                matvec of the last correction instead of
                                recomputed (counted in matvecs) */
} ibdl_solve_info;

/* Sets every field of *opts to its default. */
void ibdl_solve_opts_default(ibdl_solve_opts* opts);

/* Create a geometry handle (Sec. 5.1-5.2 inputs; the paper's "minimal
 * geometric information", Sec. 7): validates the description, copies points,
 * normals and weights, bins the points by grid tile, precomputes the delta
 * weights, the FFT twiddles and the Helmholtz symbol and allocates all
 * workspaces (grid, spectrum, Krylov basis).  Synchronises `stream` before
 * returning.  Errors: IBDL_ERR_INVALID_ARG (n not a power of two or out of
 * range, m < 1, kappa <= 0 or NaN, eta < 0 or non-finite, eta > 0 with
 * finite kappa, unknown enum, NULL pointer), IBDL_ERR_UNSUPPORTED (kappa = inf
 * with the Neumann condition),
 * IBDL_ERR_OOM, IBDL_ERR_CUDA.  *out is set only on success. */
ibdl_status ibdl_create_geometry(const ibdl_geometry_desc* desc, void* stream,
                                 ibdl_geometry* out);

/* Release a handle and its device memory (NULL is ignored).  Synchronises
 * the device first. */
void ibdl_destroy_geometry(ibdl_geometry g);

/* y = A q, one application of the boundary operator (A_D or A_N by the
 * geometry's bc), the GMRES matrix-vector product of Sec. 5.3.  q and y have
 * length m (m + 1 for a completed geometry: the operator of App. C on
 * (Q, u_bar)).  Computed in float64 for IBDL_FP64 geometries and in float32
 * (spread, FFT solve, interpolation; the +-q/2 jump in float64) for
 * IBDL_FP32_REFINED geometries.  q and y may alias. */
ibdl_status ibdl_apply(ibdl_geometry g, const double* q, double* y, void* stream);

/* Same as ibdl_apply with the precision chosen per call:
 * ibdl_precision value 0 = float64 operator, 1 = float32 operator,
 * 2 = IBDL_FP64_DF (float64 spread and interpolation, double-float
 * transforms; finite-difference, non-completed geometries, else
 * IBDL_ERR_UNSUPPORTED).  For a completed geometry (eta > 0) q and y have
 * length m + 1. */
ibdl_status ibdl_apply_precision(ibdl_geometry g, const double* q, double* y,
                                 int32_t precision, void* stream);

/* Solve the boundary system for the density (Sec. 4.1 step 1):
 *   Dirichlet: A_D Q = U_b - S* L^{-1} g~ = U_b + kappa S* L'^{-1} g~
 *   Neumann:   A_N U = S* L^{-1} S V_b - S* L^{-1} g~
 *                    = kappa S* L'^{-1} (g~ - S V_b)
 * bdata: U_b (Dirichlet) or V_b (Neumann), length m.  g_grid: optional
 * forcing g~ on the whole periodic grid (n^d values, paper convention
 * Delta u - k^2 u = g), or NULL for g = 0.  q_out: Q (Dirichlet) or the
 * unknown boundary values U (Neumann), length m.  opts/info may be NULL.
 * Synchronises `stream` (the convergence test reads residuals on the host).
 * Returns IBDL_ERR_NOT_CONVERGED with the last iterate in q_out and info
 * filled when max_iters is reached; IBDL_ERR_NONFINITE / IBDL_ERR_BREAKDOWN
 * likewise leave the last finite iterate. */
ibdl_status ibdl_solve(ibdl_geometry g, const double* bdata, const double* g_grid,
                       double* q_out, const ibdl_solve_opts* opts,
                       ibdl_solve_info* info, void* stream);

/* The grid solution (Sec. 4.1 step 2, eq. (ibdl 1 again); Neumann eq.
 * (ib neumann 1)):
 *   Dirichlet: u = kappa L'^{-1} (S~ q - g~)
 *   Neumann:   u = kappa L'^{-1} (S~ q + S vb - g~)
 * q: density from ibdl_solve (length m); vb: V_b (Neumann only, else NULL);
 * g_grid: forcing or NULL.  u_out: n^d values, x fastest.  Always float64
 * (also for FP32_REFINED geometries). */
ibdl_status ibdl_evaluate(ibdl_geometry g, const double* q, const double* vb,
                          const double* g_grid, double* u_out, void* stream);

/* Batched solves (many independent problems in one launch).  A batch object
 * owns the device descriptors of up to `capacity` (1..512) instances.
 * ibdl_solve_batched solves geoms[k] with data bdata[k] (U_b or V_b, g = 0)
 * into q_out[k] for k < count, all in ONE persistent cooperative kernel
 * launch: every instance runs the same state machine as ibdl_solve (float64
 * GMRES, or float32 GMRES cycles inside float64 residual refinement, by each
 * geometry's precision), and the resident blocks take work items (grid
 * tiles, pencils, vector chunks) of whichever instance has some, each
 * instance moving through its own phases: instances of different n, m,
 * kappa, bc and precision overlap instead of waiting for one another, and
 * finished ones drop out.  A geometry may appear once per call (its
 * workspaces hold that instance's state).  Synchronises `stream`.
 * statuses/infos (arrays of `count`, may be NULL) receive per-instance
 * results; the return value is IBDL_OK when every instance converged, else
 * the first failing instance's status. */
typedef struct ibdl_batch_s* ibdl_batch;
ibdl_status ibdl_batch_create(int32_t capacity, ibdl_batch* out);
void ibdl_batch_destroy(ibdl_batch b);
ibdl_status ibdl_solve_batched(ibdl_batch b, int32_t count, const ibdl_geometry* geoms,
                               const double* const* bdata, double* const* q_out,
                               const ibdl_solve_opts* opts, ibdl_solve_info* infos,
                               ibdl_status* statuses, void* stream);

/* Serving engine: continuous batching of independent IBDL solves.
 *
 * A server owns a table of `max_active` solver slots and a FIFO queue.
 * Requests (a geometry description with its boundary data, g = 0) are
 * submitted at any time; ibdl_server_step then
 *   1. launches one slice of the persistent solver (ibdl_solve_batched's
 *      kernel; each request runs at most `rounds_per_step` GMRES rounds in
 *      it) over every active slot -- requests of different dim, n, m, kappa, bc and
 *      precision advance together and keep their grids, spectra, FFT
 *      tables and Krylov bases resident in device memory between slices;
 *   2. while that slice runs, admits queued requests in arrival order as long
 *      as a slot is free and the device bytes of all admitted requests stay
 *      within `memory_budget`: each one's geometry is built on a second
 *      stream, on the `reserve_sms` SMs the solver leaves free, and it joins
 *      the next slice; admission stops once the slice has finished (at
 *      least one request per step), or after 8 requests when no slice runs;
 *   3. waits for the slice and retires the requests whose solve finished,
 *      releasing their slot and memory.
 * Every request is solved exactly as ibdl_solve would solve it alone (the
 * same state machine, tolerances and precision); only the scheduling is
 * shared.  This is the method's solve (Sec. 5.3) per request in serving
 * form; the paper itself has no serving counterpart.
 *
 * Thread safety: calls on one server are serialised by an internal lock.
 * Each step synchronises the server's streams. */
typedef struct ibdl_server_s* ibdl_server;

typedef struct {
  int64_t memory_budget;    /* bytes of device memory admitted requests may
                               hold; 0 = 80% of the free memory at creation */
  int32_t max_active;       /* solver slots, 1..512; default 64 */
  int32_t rounds_per_step;  /* solver rounds per request per slice, >= 1;
                               default 8 */
  int32_t reserve_sms;      /* SMs left free for request set-up while a slice
                               runs, 0..(SM count - 1); default 8 */
  int32_t reserved;
  ibdl_solve_opts opts;     /* tolerances of every request (x0 is ignored) */
} ibdl_server_config;

typedef struct {
  int64_t id;
  int32_t status;           /* ibdl_status of the solve */
  int32_t slot;
  double t_arrival;         /* seconds on ibdl_server_clock(): as submitted */
  double t_admit;           /* geometry built, slot taken */
  double t_done;            /* retired after its last slice */
  int64_t device_bytes;     /* device memory the request held */
  ibdl_solve_info info;
} ibdl_request_result;

typedef struct {
  int32_t queued, active, finished;  /* finished = completed, not yet taken */
  int32_t reserved;
  int64_t bytes_in_use, peak_bytes, memory_budget;
  int64_t steps, launches, submitted;
  double admit_seconds;     /* host time spent setting requests up */
  double wait_seconds;      /* host time spent waiting for slices */
} ibdl_server_stats;

void ibdl_server_config_default(ibdl_server_config* cfg);
/* Errors: IBDL_ERR_INVALID_ARG (bad config), IBDL_ERR_CUDA. */
ibdl_status ibdl_server_create(const ibdl_server_config* cfg, ibdl_server* out);
/* Waits for the server's streams, releases every request still held. */
void ibdl_server_destroy(ibdl_server s);
/* Monotonic clock (seconds) on which request times are measured. */
double ibdl_server_clock(void);
/* Queue a request.  desc pointers (points, normals, weights) and bdata
 * (U_b for Dirichlet, V_b for Neumann, length desc->m) may be host or device
 * memory; they are copied before the call returns.  t_arrival: the request's
 * arrival time on ibdl_server_clock() (latency is t_done - t_arrival), or a
 * negative value for "now".  Errors: IBDL_ERR_INVALID_ARG (size and pointer
 * checks of ibdl_create_geometry; the rest are made at admission, where a
 * failure finishes the request with that status), IBDL_ERR_NONFINITE
 * (bdata not finite). */
ibdl_status ibdl_server_submit(ibdl_server s, const ibdl_geometry_desc* desc,
                               const double* bdata, double t_arrival, int64_t* id_out);
/* One scheduling step (see above).  Writes up to max_ids ids of requests
 * finished in this step to done_ids (may be NULL) and their count to
 * *n_done.  Returns IBDL_OK, or IBDL_ERR_TIMEOUT / IBDL_ERR_CUDA when the
 * slice failed (the active requests are then finished with that status).
 * A request whose own solve fails, or that alone exceeds the memory budget
 * (IBDL_ERR_OOM), is finished with its status; the step still returns
 * IBDL_OK. */
ibdl_status ibdl_server_step(ibdl_server s, int64_t* done_ids, int32_t max_ids,
                             int32_t* n_done);
/* Hand over a finished request: q_out (host or device, length m, may be
 * NULL) receives its density Q (Dirichlet) or boundary values U (Neumann),
 * *res its record; the server forgets it.  IBDL_ERR_INVALID_ARG if the id
 * is unknown or not finished yet. */
ibdl_status ibdl_server_take(ibdl_server s, int64_t id, double* q_out,
                             ibdl_request_result* res);
ibdl_status ibdl_server_get_stats(ibdl_server s, ibdl_server_stats* out);

/* Component operators, exposed for testing and for callers that compose
 * their own solvers.  All float64 unless `precision` = 1.
 *   ibdl_spread_div: f = S~ q on the grid (Sec. 5.2, eq. (Stilde)).
 *   ibdl_spread:     f = S v on the grid (eq. (spread operator again2)).
 *   ibdl_helmholtz:  v = kappa L'^{-1} f (periodic FFT solve, Sec. 5.1);
 *                    f and v are n^d grids and may alias.
 *   ibdl_interp:     y = S* u at the points (eq. (interpolation again)). */
ibdl_status ibdl_spread_div(ibdl_geometry g, const double* q, double* f_out,
                            int32_t precision, void* stream);
ibdl_status ibdl_spread(ibdl_geometry g, const double* v, double* f_out,
                        int32_t precision, void* stream);
ibdl_status ibdl_helmholtz(ibdl_geometry g, const double* f, double* v_out,
                           int32_t precision, void* stream);
ibdl_status ibdl_interp(ibdl_geometry g, const double* u, double* y_out,
                        int32_t precision, void* stream);

/* Interior indicator of the discretised boundary (App. D), float64.  Solves
 * Delta_h u + S~ 1 = 0 for the mean-zero u (Q = 1, the Poisson solve
 * whatever the geometry's kappa), then
 *   chi_h = u - u(node 0)     (the box corner: far from Gamma, about 0)
 *   chi   = 1 where chi_h > 1/2, else 0
 * chi_h is about 1/2 on Gamma and about 1 inside a closed curve whose normals
 * point out of it.  chi_h_out: n^d doubles, chi_out: n^d bytes (x fastest),
 * host or device, either may be NULL (not both).  Errors:
 * IBDL_ERR_INVALID_ARG (no output), IBDL_ERR_CUDA. */
ibdl_status ibdl_indicator(ibdl_geometry g, double* chi_h_out, uint8_t* chi_out,
                           void* stream);

/* Near-boundary values (Sec. 5.5, App. A; in 3D the generalisation of
 * Sec. 6.7), float64.  u_out = u_in, except at the nodes x_p with inside = 1
 * whose nearest boundary point is closer than m1 h.  Those take the linear
 * interpolation between
 *   x_A: 2D: the orthogonal foot of x_p on the chord of its two nearest
 *        boundary points (the two of the three nearest that lie farthest
 *        apart when the foot falls outside the chord, clamped to it), with
 *        the value interpolated from ub at those two points;
 *        3D: the orthogonal foot of x_p on the plane of its three nearest
 *        boundary points, barycentric coordinates clamped to >= 0 and
 *        renormalised (the first point for a degenerate triangle), with the
 *        barycentric interpolation of ub;
 *   x_B = x_A + m2 h (x_p - x_A) / |x_p - x_A|, with the bilinear (2D) or
 *        trilinear (3D) interpolation of u_in in its grid cell.
 * Ties in distance go to the lower point index.  ub: the boundary values
 * (U_b for Dirichlet, the solved U for Neumann), length m.  inside: n^d
 * bytes, 1 = node of Omega (e.g. ibdl_indicator's chi, or 1 - chi for an
 * exterior domain).  u_in, u_out: n^d doubles (x fastest), must not
 * overlap.  All host or device.  m1 in 1..n/2 (the paper uses 6), m2 > 0
 * (the paper uses m1 + 2).  Errors: IBDL_ERR_INVALID_ARG (m < 3, m1 or m2
 * out of range, NULL or overlapping arrays), IBDL_ERR_CUDA. */
ibdl_status ibdl_near_boundary(ibdl_geometry g, const double* u_in, const double* ub,
                               const uint8_t* inside, int32_t m1, double m2, double* u_out,
                               void* stream);

/* Self-test of the bounded device waits that the persistent solver uses
 * between its blocks.  One block joins a barrier of two parties, so its
 * wait cannot complete; it gives up after spin_limit polls (1 .. 2^24; the
 * solver's own limit is 2^27), raises the error word and returns.  Returns
 * IBDL_ERR_TIMEOUT when the wait gave up as designed (the context stays
 * usable), IBDL_OK if it did not, IBDL_ERR_INVALID_ARG, IBDL_ERR_CUDA. */
ibdl_status ibdl_selftest_bounded_wait(uint32_t spin_limit, void* stream);

/* Read-only facts about a handle. */
typedef struct {
  int32_t dim, n;
  int64_t m;
  double h, kappa;
  int32_t bc, delta, precision;
  int64_t device_bytes;      /* device memory the handle owns */
  int32_t fft_passes;        /* kernels per Helmholtz solve */
  int32_t rows_per_tile;     /* grid rows per x-pass tile (spread bin size) */
  int32_t pencils_per_item[2]; /* pencils per work item of the solve pass (2D y,
                                  3D z) and of the 3D y passes (0 in 2D), in
                                  the geometry's inner precision */
  int32_t fft_plan;          /* FFT plan variant of the float32 transforms:
                                0 radices as even as possible after a first
                                radix-16 pass (1024 = 16*8*8), 1 radix-16
                                passes first (1024 = 16*16*4; n = 512, 1024) */
} ibdl_geometry_info;
ibdl_status ibdl_get_geometry_info(ibdl_geometry g, ibdl_geometry_info* info);

/* Autotuner of the x-pass tiling and of the pencil items (on by default).
 * The first geometry of each (device, dim, n, precision) times one matvec
 * for every admissible number of grid rows per tile -- an even R with
 * n/R >= 4, R <= n - 5 and float64 row buffers within 100 KB of shared
 * memory -- then, with that tiling, for every admissible number of pencils
 * per work item of each pencil pass (a power of two <= 16 whose item fits
 * 100 KB; strided z items at least 2), in the geometry's inner precision; the
 * fastest choices are used by every later geometry of that kind in the
 * process (a few matvecs once, inside that first ibdl_create_geometry).
 * The pencil choice applies to the launch-based passes (ibdl_apply,
 * ibdl_evaluate, ibdl_helmholtz, the host-loop engine); the persistent
 * solver keeps the fixed rule, under which its instances share the GPU
 * better.  Geometries built by the
 * server use a tiling already chosen, else the fixed rule (4 rows in 2D, 2
 * for n = 2048; 8 in 3D).  Off: the fixed rule always.  Results of the two
 * tilings agree to rounding. */
void ibdl_tuning_enable(int32_t on);

/* Pins the x-pass tiling of one (current device, dim, n, precision): later
 * geometries of that kind use `rows` grid rows per tile, as if the tuner
 * had chosen it (while tuning is on; off, the fixed rule applies).  rows = 0
 * drops the entry, so the next geometry of the kind tunes again.  For
 * reproducible launches (a deployment that fixes its configuration, or a
 * profiler run, under which timing candidates would be distorted).
 * IBDL_ERR_INVALID_ARG unless dim is 2 or 3, n a power of two in
 * [16, 2048] (2D) / [16, 512] (3D), precision a geometry's (IBDL_FP64 or IBDL_FP32_REFINED),
 * and rows 0 or an admissible tiling (as above); IBDL_ERR_CUDA if the current device cannot be read. */
ibdl_status ibdl_tuning_set(int32_t dim, int32_t n, int32_t precision, int32_t rows);

/* Pins the pencils per work item of one (current device, dim, n,
 * precision) kind, as if the autotuner had chosen them: c_solve for the solve
 * pass (2D y pencils, 3D z pencils), c_y for the 3D y passes (0 in 2D); 0 for
 * one of them keeps the fixed rule for that pass, and both 0 drops the entry
 * (the next geometry of the kind tunes again).  The precision's own element
 * type is pinned (float32 for IBDL_FP32_REFINED, float64 for IBDL_FP64); a
 * value must be admissible: a power of two <= 16 whose item fits 100 KB of
 * shared memory, at least 2 and at most n for strided z pencils.  Later
 * geometries of the kind use the pin; results agree with the fixed rule's to
 * rounding.  IBDL_ERR_INVALID_ARG otherwise; IBDL_ERR_CUDA if the current
 * device cannot be read.  No passage of the paper: a resource choice. */
ibdl_status ibdl_tuning_set_pencils(int32_t dim, int32_t n, int32_t precision, int32_t c_solve,
                                    int32_t c_y);

/* Pins the FFT plan variant of the float32 transforms of one (current
 * device, dim = 2, n, IBDL_FP32_REFINED) kind, as if the autotuner had
 * chosen it:
 * plan 0 = a first pass of radix 16, then the remaining bits split as evenly
 * as possible (1024 = 16 * 8 * 8, 512 = 16 * 8 * 4); plan 1 = radix-16
 * passes first, the remainder last (1024 = 16 * 16 * 4, 512 = 16 * 16 * 2),
 * offered for n = 512 and 1024 only (the other sizes have one plan); plan -1
 * drops the pin (the next geometry of the kind tunes again; 3D geometries
 * always use plan 0).  Later geometries of the
 * kind transform in that plan everywhere in float32, the persistent solver
 * included; results agree with plan 0's to rounding.  IBDL_ERR_INVALID_ARG
 * for another precision, size or plan; IBDL_ERR_CUDA if the current device
 * cannot be read.  No passage of the paper: a resource choice. */
ibdl_status ibdl_tuning_set_plan(int32_t dim, int32_t n, int32_t precision, int32_t plan);

/* Pencils per work item of the persistent solver's solve pass (2D y
 * pencils, 3D z pencils) for this geometry's solves, per element type:
 * c_f64 float64, c_f32 float32 (the refined inner operator), c_dd
 * double-float (the residuals of small refined launches); 0 keeps the fixed
 * rule (every y or z pencil group of about 256 items).  Fewer, larger items
 * let the instances of one batched launch run side by side; more, smaller
 * ones shorten a lone solve's phases.  Each value must be admissible (a
 * power of two <= 16 whose item fits 100 KB of shared memory; strided z
 * items at least 2), and the solver's items must fit one block's shared
 * memory.  Results agree with the fixed rule's to rounding.
 * IBDL_ERR_INVALID_ARG otherwise (the geometry is left as it was).  No
 * passage of the paper: a resource choice. */
ibdl_status ibdl_geometry_set_solver_pencils(ibdl_geometry g, int32_t c_f64, int32_t c_f32,
                                             int32_t c_dd);

/* Shared-memory bookkeeping of the persistent solver's work items (host
 * only: touches no GPU, so it runs without one).  For a grid (dim, n), an
 * x-pass tiling of `rows` grid rows per tile (a power of two in [2, n]) and
 * an element type elem (0 float64, 1 float32, 2 double-float), with n a
 * power of two in [16, 2048] (2D) / [16, 512] (3D), need_out[0]
 * receives the dynamic shared memory of one x-pass row tile, need_out[1] of
 * one item of the solve pencil pass (2D: y pencils; 3D: z pencils) and
 * need_out[2] of one item of the 3D y pencil passes (0 in 2D); budget_out
 * the dynamic shared memory a solver launch over such a geometry reserves
 * (the largest need over the element types the solve can run), and
 * twiddles_out the entries of the FFT's twiddle table.  Any output may be
 * NULL.  A launch checks the same figures for every instance before it
 * starts and returns IBDL_ERR_INVALID_ARG instead of launching when an item
 * would not fit.  IBDL_ERR_INVALID_ARG for unsupported sizes.  No passage of
 * the paper: this is the library's own resource accounting. */
ibdl_status ibdl_solver_smem_query(int32_t dim, int32_t n, int32_t rows, int32_t elem,
                                   int64_t need_out[3], int64_t* budget_out,
                                   int32_t* twiddles_out);

/* Number of this library's kernels launched so far in this process
 * (all handles, all streams). */
int64_t ibdl_kernel_launch_count(void);

/* Kernel timing (off by default).  While on, every launch of this library is
 * bracketed by a pair of CUDA events recorded on its own stream; the pairs
 * are resolved by ibdl_profile_read.  The events add a few microseconds of
 * host work per launch, so time end-to-end figures with profiling off. */
void ibdl_profile_enable(int32_t on);

typedef struct {
  char name[48];       /* kernel family, e.g. "rows_fwd_f64", "pencils_solve_f32" */
  int64_t launches;
  double total_ms;     /* summed event-measured duration */
} ibdl_kernel_stat;

/* Synchronises the device, folds all pending event pairs into per-kernel
 * totals and copies up to max_out entries (sorted by name) to out (may be
 * NULL).  Returns the number of kernel families recorded; reset != 0 clears
 * the totals afterwards. */
int32_t ibdl_profile_read(ibdl_kernel_stat* out, int32_t max_out, int32_t reset);

/* Work-item trace of the persistent solver (diagnostics; needs profiling
 * on).  On clears the trace; while on, each block of a persistent launch
 * writes one record per work item it runs and one per phase hand-off, into
 * its own share of 65536 records (later records of a block whose share is
 * full are dropped).  IBDL_ERR_INVALID_ARG if profiling is off. */
ibdl_status ibdl_profile_trace(int32_t on);

/* Synchronises the device, copies up to max_records trace records (three
 * uint64 words each: start and end on the GPU's global nanosecond timer, then
 * block << 40 | instance << 24 | phase << 20 | precision << 18 | item, where
 * phase 0..4 are the matvec phases (x forward, 3D y forward, solve, 3D y
 * inverse, x inverse), 5..9 the vector phases and the one-block step, 15 a
 * hand-off whose item field is the next phase (15: the instance stopped), and
 * precision 1 float32 items) to out (may be NULL), then clears the trace.
 * Returns the number of records written since the trace was last cleared,
 * or -1 on a CUDA error. */
int64_t ibdl_profile_trace_read(uint64_t* out, int64_t max_records);

/* Allocation-free variant of ibdl_helmholtz for callers that cannot
 * allocate device memory: code running inside a host callback or a stream
 * callback, or a plugin whose host application owns every device
 * allocation, where a cudaMalloc is forbidden, would deadlock or would grow
 * a footprint that must stay fixed after start-up.  The paper has no
 * counterpart.
 *
 * Computes v_out = kappa L'^{-1} f on an n x n periodic grid of spacing
 * h = box_len / n (L' = I - kappa Delta_h, 5-point stencil), float64, exactly
 * as ibdl_helmholtz does, without a geometry handle.  f and v_out are n*n
 * float64 values in DEVICE memory (x fastest) and may alias.  n must be a
 * power of two in [16, 512]; larger n returns IBDL_ERR_INVALID_ARG with a
 * message naming the limit.
 *
 * Scratch: one file-scope __device__ array of about 2.1 MB (a 512 x 512
 * half spectrum, twiddle and symbol tables) that every GPU loading the
 * library holds until the process exits.  After the first call on a device
 * the call allocates nothing and calls no allocating routine.  The FIRST
 * call on each device is set-up: it looks up the array's device address with
 * cudaGetSymbolAddress (with that device current), and under CUDA's lazy
 * module loading it is also the call that loads this part of the library,
 * which places the static array and the kernels in device memory.  Make that
 * first call at start-up, where allocation is allowed, and before any stream
 * capture.  Every call shares the array and rewrites the parts it reads
 * (tables, tile lists, spectrum), so calls that overlap on the GPU -- on
 * different streams or from different host threads -- race and must be
 * serialised by the caller.  Asynchronous on `stream`. */
ibdl_status ibdl_helmholtz_2d_noalloc(int32_t n, double box_len, double kappa,
                                      const double* f, double* v_out, void* stream);

const char* ibdl_status_string(ibdl_status s);
const char* ibdl_last_error_message(void);
int32_t ibdl_version(void); /* 100 * MAJOR + MINOR */

#ifdef __cplusplus
}
#endif
#endif /* IBDL_H_ */
