/*
 * ls.h -- C ABI of the GB300 Lippmann-Schwinger forward model and gradient.
 *
 * Implements the discrete model of Pham et al., "Three-Dimensional Optical
 * Diffraction Tomography with Lippmann-Schwinger Model" (arXiv 1910.13844):
 *
 *   eq. lipp1   u    = (I - G diag(f))^{-1} u_in            (BiCGStab, Sec. 2.2)
 *   eq. lipp2   y_sc = G~ diag(f) u                          (P = I)
 *   Alg. 1 l.6  grad = sum_q c_q Re(conj(u_q) .* w_q),
 *               (I - G^H diag(f)) w_q = G~^H r_q             (Sec. 4.2)
 *
 * G is the Vainikko discretisation of the truncated Green function
 * (Theorem 1) applied with twofold zero padding through the modified kernel
 * of Proposition 1; G~ is the detector-plane operator of eq. Gtild-1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.  Volumes are [nz][ny][nx] row-major (x fastest).  Voxel (i, j, k)
 *   (x, y, z array indices) sits at h * (i - nx/2 + 1, j - ny/2 + 1,
 *   k - nz/2 + 1) micrometres: the centred index set of Sec. 1.4.  The
 *   detector is [my][mx], pixel (a, b) (row, column) at
 *   (h (b - mx/2 + 1), h (a - my/2 + 1), x_gamma).
 * Types.  ls_c64 is interleaved complex64 (8 bytes); potentials and
 *   gradients are float32.  Reductions inside the solver run in float64.
 * Memory.  Every ls_c64/float pointer is DEVICE memory owned by the caller
 *   unless stated otherwise; "host" marks host pointers.  Arrays of pointers
 *   (const ls_c64* const* u_in, ...) are HOST arrays of n_views device
 *   pointers, one per view.  The library never frees caller memory.  The plan
 *   owns the Green spectrum, the far-field kernels and the solver workspace.
 * Streams.  cuda_stream is a cudaStream_t (NULL = legacy default stream).
 *   Calls enqueue work on it; calls that return solver statistics
 *   synchronise it before returning.
 * Errors.  Every int-returning call returns LS_OK (0) or one of the LS_E*
 *   codes below.  Nothing is thrown across the ABI.  ls_last_error() gives
 *   a thread-local message for the last failure.
 * Threads.  One plan must not be used by two threads at once.
 */
#ifndef LS_H
#define LS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

enum ls_status {
  LS_OK = 0,
  LS_EINVAL = 1,         /* bad argument (size, pointer, option); nothing was enqueued   */
  LS_ENOMEM = 2,         /* a device allocation failed                                    */
  LS_ECUDA = 3,          /* a CUDA runtime call failed; see ls_last_error()               */
  LS_NOT_CONVERGED = 4,  /* max_iter reached; outputs written, stats say which view        */
  LS_BREAKDOWN = 5,      /* BiCGStab breakdown (rho or <r0,v> vanished) after all restarts */
  LS_TIMEOUT = 6,        /* a solve's bounded host loop ended with views still running    */
  LS_PENDING = 7,        /* ls_poll: request not finished yet                              */
  LS_EAGAIN = 8,         /* ls_submit: the request can never fit the server's HBM budget   */
  LS_ENOTFOUND = 9,      /* ls_poll: unknown or already collected ticket                   */
  LS_EUNSUPPORTED = 10   /* grid size with no FFT length implemented (see ls_grid)         */
};

typedef struct { int nx, ny, nz; } ls_grid;      /* voxels per axis, each in {8,12,16,24,32,48,64,72,96,128,144,192} */
typedef struct { float re, im; } ls_c64;

typedef struct {
  double tol;          /* BiCGStab stop: ||r|| <= tol ||b|| (recursive residual).  Default 1e-6.      */
  int max_iter;        /* iterations per view before LS_NOT_CONVERGED.  Default 1000.                 */
  int oversample_p;    /* Green-spectrum oversampling p of Theorem 1 / Prop. 1 (even, >= 2).  Default 4 */
  int det_mx, det_my;  /* detector pixels (0 = nx, ny); m <= n and n - m even (centred window).     */
  double x_gamma;      /* detector plane position along z in micrometres; <= 0 means 3 L_z / 4.       */
  int max_restarts;    /* restarts from the true residual when it misses 10 tol at exit.  Default 4.  */
  int check_every;     /* iterations between host reads of the convergence mask (0 = 2).             */
  int use_graphs;      /* 1 = replay the BiCGStab iteration from a captured CUDA graph.  Default 1.  */
  double cone_sin_theta; /* built-in illumination (u_in == NULL): view q of n is the plane wave of wave   */
                         /* vector k_b (s cos phi_q, s sin phi_q, sqrt(1 - s^2)), s = cone_sin_theta     */
                         /* (= NA / eta_b), phi_q = 2 pi q / n (the cone of Fig. 1).  Default 0 (+z).    */
} ls_options;

typedef struct {
  int status;                 /* LS_OK, LS_NOT_CONVERGED, LS_BREAKDOWN or LS_TIMEOUT             */
  int iterations;             /* BiCGStab iterations (each has two matvecs)                      */
  int restarts;               /* restarts from the true residual                                 */
  int matvecs;                /* operator applications including residual checks                 */
  double rel_residual;        /* recursive ||r|| / ||b|| at exit                                 */
  double true_rel_residual;   /* recomputed ||b - A x|| / ||b|| at exit (float32 operator)       */
} ls_stats;

typedef struct ls_plan ls_plan;

/* Launch variants chosen by ls_autotune (no counterpart in the paper). */
typedef struct {
  int z_tma;              /* 1: TMA-staged z pass with warp-local exchanges; 0: cp.async-staged            */
  int ix_prefetch;        /* 1: the last pass asks L2 for its epilogue operands at kernel start            */
  int fx_views_fastest;   /* 1: first-pass grid with the views fastest (shared potential rows from L2)      */
  int check_every;        /* BiCGStab iterations between host reads of the convergence mask                */
  int use_graphs;         /* 1: iterations replayed from a captured CUDA graph                              */
  double matvec_us_per_view;  /* batched operator application with the chosen variants, per view (µs)      */
  double solve_ms;            /* forward solve of the tuning batch with the chosen variants (ms)            */
  int from_cache;             /* 1: read from the LS_AUTOTUNE_CACHE file, nothing was timed                  */
  int z_split;                /* 1: the TMA-staged z pass with its second radix split                          */
  int strided_wide;           /* 1: the y passes with 32 pencils per CTA (else 16)                             */
  int views_per_launch;       /* BiCGStab iteration launched over chunks of this many views (0: all at once)   */
  int z_persist;              /* TMA-staged z pass: 0 one CTA per tile; persistent (one wave of CTAs):         */
                              /*   1 tiles assigned round-robin, 2 work units (a tile, a chunk of its views)   */
                              /*   taken from a counter                                                       */
  int fx_bulk;                /* 1: the first pass with bulk-copy-staged input rows (persistent)              */
} ls_tune;

/* Fill *opt with the defaults listed above. */
void ls_default_options(ls_options* opt);

/* Create a plan for one grid: voxel pitch `voxel` (um, = h of Theorem 1),
 * background wavenumber k_b = 2 pi eta_b / lambda (1/um, Sec. 2.1).
 * `padding` is the storage padding of Prop. 1 and must be 2.  Builds the
 * Green spectrum with opt->oversample_p (see ls_green_spectrum) and the
 * far-field kernels (Sec. 3.2).  Requires k_b h < pi (Theorem 1).  *out
 * receives the plan, to be released with ls_plan_destroy.  Errors:
 * LS_EINVAL, LS_EUNSUPPORTED, LS_ENOMEM, LS_ECUDA. */
int ls_plan_create(const ls_grid* grid, int padding, double k_b, double voxel,
                   const ls_options* opt, ls_plan** out);
void ls_plan_destroy(ls_plan* plan);

/* (Re)build the Green spectrum Ghat = F_{2n}(g_t^m) of Prop. 1 for
 * oversampling p (even >= 2): ghat_t of eq. GreenL/GreenL2 sampled at
 * delta ((p/2) q - s), (p/2)^3 inverse FFTs of size (2n)^3, phase-shifted sum,
 * kernel zeroed at the Nyquist offset, forward FFT -- all in float64 on the
 * GPU, then stored as complex64 (one octant, Ghat is even in every axis).
 * If out_full != NULL it receives the full spectrum, (2nz)(2ny)(2nx) ls_c64,
 * unnormalised (the same array as F_{2n} of the kernel).  Synchronous. */
int ls_green_spectrum(ls_plan* plan, int oversample_p, ls_c64* out_full, void* cuda_stream);

/* Scattering potential f = k_b^2 ((eta_b + dn)^2 / eta_b^2 - 1) (Sec. 2.1)
 * for `count` voxels: dn (device float32 contrast) -> f (device float32). */
int ls_scattering_potential(const float* dn, size_t count, double eta_b, double k_b,
                            float* f, void* cuda_stream);

/* Incident plane waves u_in,q(x) = exp(i k_q . x) at the voxel centres
 * (Fig. 1).  kvec: host array of 3 * n_views doubles (kx, ky, kz per view,
 * 1/um).  u_in[q]: device, N complex64 each. */
int ls_plane_waves(ls_plan* plan, int n_views, const double* kvec,
                   ls_c64* const* u_in, void* cuda_stream);

/* out = G v (adjoint != 0: G^H v), Theorem 1 with Prop. 1's kernel.  v, out: N complex64. */
int ls_apply_green(ls_plan* plan, const ls_c64* v, ls_c64* out, int adjoint, void* cuda_stream);

/* y = x - G (f .* x) (adjoint != 0: x - G^H (f .* x)), the operator of eq. lipp1. */
int ls_matvec(ls_plan* plan, const float* f, const ls_c64* x, ls_c64* y, int adjoint,
              void* cuda_stream);

/* y[q] = x[q] - G (f .* x[q]) (adjoint != 0: with G^H) for n_views vectors at
 * once: every FFT pass is one launch over all vectors (the batched form the
 * solver uses).  x, y: host arrays of n_views device pointers (N complex64
 * each; y[q] may equal x[q]). */
int ls_matvec_batch(ls_plan* plan, const float* f, int n_views, const ls_c64* const* x, ls_c64* const* y,
                    int adjoint, void* cuda_stream);

/* Same operator as ls_matvec (y = x - G (f .* x), or with G^H), for callers
 * that cannot allocate device memory: a process whose device memory is all
 * owned by its own pool, or a loop that must not stall on the implicit device
 * synchronisation of cudaMalloc/cudaFree.  ls_matvec may allocate the plan's
 * workspace on first use; this call allocates nothing.  Its FFT
 * intermediates live in one static device array of 64 MiB inside the library
 * (48 bytes per voxel: grids up to 1398101 voxels, e.g. 96^3 or 128x128x64).
 * The array is reserved on a device, and its device address looked up, by the
 * first ls_plan_create on that device (which allocates anyway); it is then
 * held until the process exits.  So create the plan before handing the rest of
 * the device's memory to a pool; this call itself looks nothing up, loads
 * nothing and allocates nothing, on its first use too.  It must run on the
 * device the plan was created on (LS_EINVAL otherwise).  Larger grids return
 * LS_EINVAL with the sizes in ls_last_error().  All calls share the one array:
 * calls that overlap on the GPU (different streams, or different host
 * threads) race and must be ordered by the caller.  Nothing has to be cleared
 * between calls.  The paper has no counterpart to this entry point. */
int ls_matvec_noalloc(const ls_plan* plan, const float* f, const ls_c64* x, ls_c64* y, int adjoint,
                      void* cuda_stream);

/* Forward model for n_views illuminations of one potential f (eqs. lipp1, lipp2):
 * BiCGStab on (I - G diag f) u = u_in[q] from u = u_in[q], all views batched,
 * then the far field y_q = G~ (f .* u_q) on the detector.  u_in == NULL: the
 * plan's built-in plane waves (ls_options.cone_sin_theta), generated in the
 * solver's workspace (no caller buffer, no copies).  u_out[q] (N) and
 * far[q] (my*mx) may each be NULL (u_out == NULL: fields not returned;
 * far == NULL: far field skipped).  stats: host array of n_views or NULL.
 * Returns LS_OK, LS_NOT_CONVERGED, LS_BREAKDOWN or LS_TIMEOUT (worst view), or an error;
 * LS_ECUDA also when a z-pass wait on its own TMA copy gave up (bounded, one second). */
int ls_forward(ls_plan* plan, const float* f, int n_views, const ls_c64* const* u_in,
               ls_c64* const* u_out, ls_c64* const* far, ls_stats* stats, void* cuda_stream);

/* ls_forward with initial guesses: BiCGStab for view q starts from x0[q] (device, N complex64
 * each; may alias u_out[q]) instead of u_in[q].  Used to warm-start the forward solves of one
 * reconstruction iteration from the fields of the previous one (Alg. 1 evaluates the model at
 * potentials that change little between iterations); the paper states no initial guess. */
int ls_forward_warm(ls_plan* plan, const float* f, int n_views, const ls_c64* const* u_in,
                    const ls_c64* const* x0, ls_c64* const* u_out, ls_c64* const* far, ls_stats* stats,
                    void* cuda_stream);

/* far[q] = G~ (f .* u[q]) (eq. Gtild-1, midpoint rule, exact per-slice 2-D convolutions). */
int ls_farfield(ls_plan* plan, const float* f, int n_views, const ls_c64* const* u,
                ls_c64* const* far, void* cuda_stream);

/* out[q] = G~^H r[q]: r[q] is my*mx, out[q] is N. */
int ls_farfield_adjoint(ls_plan* plan, int n_views, const ls_c64* const* r,
                        ls_c64* const* out, void* cuda_stream);

/* Pupil / refocus operator P of eq. lipp2 (Sec. 3.3): a convolution on the detector applied by FFT
 * on the detector zero-padded to 2my x 2mx, with transfer function
 *   H(w) = 1{|w| <= k_cut} exp(i distance sqrt(k_b^2 - |w|^2))   (evanescent components dropped):
 * an ideal pupil of cut-off k_cut (1/um, e.g. 2 pi NA / lambda) and a free-space propagation over
 * `distance` um (e.g. the refocus from the detector plane to the sample centre, -x_gamma).
 * Once set, ls_forward / ls_farfield return P G~ (f u) and ls_gradient / ls_farfield_adjoint apply
 * G~^H P^H.  k_cut <= 0 removes the pupil (P = I, the default).  Synchronous; computed in float64. */
int ls_set_pupil(ls_plan* plan, double k_cut, double distance);
/* out[q] = P in[q] (adjoint != 0: P^H in[q]); in, out: my*mx complex64 each (may alias). */
int ls_apply_pupil(ls_plan* plan, int n_views, const ls_c64* const* in, ls_c64* const* out, int adjoint,
                   void* cuda_stream);

/* x = prox_{lam TV + i_{>=0}}(z) = argmin_{x >= 0} 0.5 ||x - z||^2 + lam TV(x), the prox step of
 * Alg. 1 (Sec. 4.2) with the isotropic total variation (forward differences, zero difference on the
 * last plane of each axis), evaluated by `iters` iterations of the fast gradient projection method
 * on the dual (step 1/(12 lam)), as the paper does.  z, x: device float [nz][ny][nx] that must not
 * overlap when lam > 0; work: device scratch of 6*nx*ny*nz floats, or NULL to allocate it on the
 * stream.  lam <= 0 gives max(z, 0) (then z and x may alias).  Asynchronous on cuda_stream. */
int ls_prox_tv(const ls_grid* grid, const float* z, float* x, double lam, int iters, float* work,
               void* cuda_stream);

/* x = argmin_{x >= 0} 0.5 ||x - z||^2 + lam sum_v ||H x (v)||_{S1}: the prox step of Alg. 1 with the
 * Hessian Schatten-norm regulariser (Sec. 4.2), H the discrete Hessian (second differences D_aa =
 * -D_a^T D_a with a Neumann boundary, mixed D_ab = D_b D_a of forward differences), ||.||_{S1} the
 * nuclear norm of each voxel's symmetric 3 x 3 Hessian; evaluated by `iters` FGP iterations on the
 * dual (spectral-norm ball per voxel, step 1/(144 lam)).  z, x: device float [nz][ny][nx] that must
 * not overlap when lam > 0; work: device scratch of 12*nx*ny*nz floats, or NULL to allocate it on the
 * stream.  lam <= 0 gives max(z, 0).  Asynchronous on cuda_stream. */
int ls_prox_hs(const ls_grid* grid, const float* z, float* x, double lam, int iters, float* work,
               void* cuda_stream);

/* Times the launch variants of ls_tune on this plan's grid with n_views plane-wave views of the
 * potential f (device, N floats), one knob after the other, and keeps the fastest in the plan (the
 * plan's check_every / use_graphs options are overwritten).  If the environment variable
 * LS_AUTOTUNE_CACHE names a file, a result for the same device, grid and view count is read from it
 * instead of timing, and new results are appended to it.  The z-pass form chosen applies to launches
 * of more than n_views / 2 views; smaller batches on the same plan keep the per-length default form
 * (the fastest form depends on the batch size).  Synchronous; uses the plan's workspace (its
 * contents are overwritten).  out may be NULL.  No counterpart in the paper. */
int ls_autotune(ls_plan* plan, int n_views, const float* f, ls_tune* out, void* cuda_stream);

/* Incident fields from their measurement on the detector plane (Sec. 3.4): for every plane z of
 * the volume, u_in(., z) = p_z * y_in with p_hat_z(w) = exp(-i (x_gamma - z) sqrt(k_b^2 - |w|^2))
 * (eq. propUin; evanescent components dropped), computed as a periodic convolution on the
 * ny x nx lateral grid.  With k_in (host, 2 doubles per view: the lateral wave vector of the
 * illumination) the tilt transfer of eq. propUin-2 is used: y_in = a exp(i x.k_in), the shifted
 * kernel p_hat_z(w + k_in) is applied to the amplitude a and the tilt is multiplied back; k_in ==
 * NULL propagates y_in directly.  y_in[q]: device ny*nx complex64 (the detector sampled on the
 * volume's lateral grid at z = x_gamma); u_in[q]: device N complex64.  Computed in float64. */
int ls_incident_field(ls_plan* plan, int n_views, const ls_c64* const* y_in, const double* k_in,
                      ls_c64* const* u_in, void* cuda_stream);

/* res[q] = pred[q] - meas[q] over `count` complex entries per view, and
 * loss_out[q] (host, may be NULL) = ||res[q]||^2 accumulated in float64. */
int ls_residual(int n_views, size_t count, const ls_c64* const* pred, const ls_c64* const* meas,
                ls_c64* const* res, double* loss_out, void* cuda_stream);

/* Data-fidelity gradient (Alg. 1 line 6, Jacobian adjoint):
 *   grad = sum_q c_q Re(conj(u_q) .* w_q),  (I - G^H diag f) w_q = G~^H r_q,
 * with r_q = residuals[q] (my*mx, e.g. H_q(f) - y_q) and c_q = view_weights[q]
 * (host array; NULL means 1; double where the paper's c_q = 1/||y_q||^2 can span
 * many decades).  u_fwd[q] are the forward fields (checkpoint); if u_fwd == NULL
 * they are recomputed from u_in (NULL: the built-in plane waves, as in
 * ls_forward); u_in is ignored otherwise.
 * grad: N float32, overwritten.  stats: host array of n_views (adjoint solves) or NULL. */
int ls_gradient(ls_plan* plan, const float* f, int n_views, const ls_c64* const* u_in,
                const ls_c64* const* u_fwd, const ls_c64* const* residuals,
                const double* view_weights, float* grad, ls_stats* stats, void* cuda_stream);

/* <a[q], b[q]> = sum_i conj(a[q][i]) b[q][i] over `count` entries for each of n_views pairs: the inner
 * product of BiCGStab's scalars (Sec. 2.2), evaluated the way the solver's kernels evaluate theirs
 * (float32 products and per-thread partial sums, every sum across threads in float64, fixed order).
 * out: host array of 2 * n_views doubles (re, im per view).  Synchronous on cuda_stream. */
int ls_inner_products(int n_views, size_t count, const ls_c64* const* a, const ls_c64* const* b, double* out,
                      void* cuda_stream);

/* ---------------------------------------------------------------- serving */

enum ls_request_kind { LS_REQ_FORWARD = 0, LS_REQ_GRADIENT = 1 };

typedef struct {
  size_t hbm_budget_bytes;   /* device memory the server may use for plans and Krylov state (0 = 80% of free) */
  int max_views_per_grid;    /* cap of concurrently resident views per grid size (0 = no cap)                  */
  double tol;                /* solver tolerance (0 = 1e-6)                                                     */
  int max_iter;              /* 0 = 1000                                                                        */
  double k_b, voxel;         /* optics shared by all requests (1/um, um)                                        */
  int iters_per_round;       /* BiCGStab iterations a lane runs between reads of its slot states (0 = 2)       */
} ls_server_options;

typedef struct {
  int kind;                  /* LS_REQ_FORWARD or LS_REQ_GRADIENT                                   */
  ls_grid grid;              /* voxel counts                                                        */
  int n_views;
  const float* f;            /* device, N; must stay valid until ls_poll returns a final status     */
  const double* kvec;        /* host, 3*n_views plane-wave vectors (copied by ls_submit)            */
  const ls_c64* meas;        /* GRADIENT: device [n_views][my*mx] measurements y_q                   */
  ls_c64* u_out;             /* device [n_views][N] or NULL                                         */
  ls_c64* far;               /* device [n_views][my*mx] or NULL (FORWARD)                            */
  float* grad;               /* GRADIENT: device N, gradient of sum_q ||H_q - y_q||^2/(2||y_q||^2) */
  double* loss;              /* GRADIENT: host double receiving the loss, or NULL                    */
} ls_request;

typedef struct {
  int status;                /* final status of the request (LS_OK, LS_NOT_CONVERGED, ...)         */
  int iterations_max;        /* largest BiCGStab iteration count over the request's views          */
  double submit_to_done_ms;  /* wall time from ls_submit to completion                             */
} ls_result;

typedef struct ls_server ls_server;

/* Start a server thread that runs continuous batching: requests of the same
 * grid share one batched BiCGStab engine; new requests join at iteration
 * boundaries as slots and device memory free up. */
int ls_server_create(const ls_server_options* opt, ls_server** out);
/* Queue a request (copied; device buffers are referenced).  *ticket identifies it.
 * LS_EAGAIN if it can never fit the HBM budget, LS_EINVAL on bad arguments. */
int ls_submit(ls_server* srv, const ls_request* req, uint64_t* ticket);
/* LS_PENDING while running; otherwise the final status (also in res) and the
 * ticket is released.  res may be NULL. */
int ls_poll(ls_server* srv, uint64_t ticket, ls_result* res);
/* Stops the server thread after the queued work and frees its memory. */
void ls_server_destroy(ls_server* srv);

/* ---------------------------------------------------------------- profiling */

/* Kernel kinds timed by ls_profile (the five FFT passes of one operator
 * application, the BiCGStab update and scalar steps, far-field kernels). */
enum ls_kernel_kind {
  LS_K_FX = 0, LS_K_FY = 1, LS_K_Z = 2, LS_K_IY = 3, LS_K_IX = 4,
  LS_K_UPDATE = 5, LS_K_SCALAR = 6, LS_K_FAR = 7, LS_K_OTHER = 8, LS_K_COUNT = 9
};

typedef struct {
  double ms[LS_K_COUNT];          /* summed device time per kind (CUDA events around each launch) */
  long long launches[LS_K_COUNT]; /* launches per kind                                            */
  long long slot_passes[LS_K_COUNT]; /* sum over launches of the slots each launch covered        */
  long long active_slot_passes[LS_K_COUNT]; /* slots that actually ran (not masked off), summed     */
} ls_kernel_times;

/* enable = 1: reset the counters and time every kernel launch of this plan
 * with a CUDA event pair on the launching stream (graph replay is disabled
 * while profiling so each launch can be bracketed).  enable = 0: stop.
 * out (host, may be NULL) receives the totals so far (synchronises the plan's
 * pending events).  Adds no work to the kernels themselves. */
int ls_profile(ls_plan* plan, int enable, ls_kernel_times* out);

/* ---------------------------------------------------------------- failure injection (tests) */

/* Test-only failure injection, for checking the library's failure paths without faulting a GPU (the
 * paper has no counterpart).  Every kind is off by default; LS_INJECT_NONE clears them all. */
enum ls_inject_kind {
  LS_INJECT_NONE = 0,         /* plan: clear every injection of this plan and the allocation counter      */
  LS_INJECT_ZERO_SHADOW = 1,  /* plan: view `value` gets a zero shadow residual at the start of each solve, */
                              /*   so <rh, v> vanishes in its first iteration (a forced BiCGStab breakdown;  */
                              /*   a restart from the true residual recovers it); value < 0 turns it off    */
  LS_INJECT_MAX_ROUNDS = 2,   /* plan: a solve's host loop stops after `value` rounds of launches; views    */
                              /*   still running report LS_TIMEOUT; value < 0 restores the normal bound     */
  LS_INJECT_ALLOC_FAIL = 3,   /* process-wide (plan may be NULL): the next `value` solver-workspace         */
                              /*   allocations (plans and server lanes) fail with LS_ENOMEM                  */
  LS_INJECT_Z_STALL = 4,      /* plan: value > 0: the TMA-staged z pass waits on a barrier that nothing     */
                              /*   completes and gives up after `value` ns (every copy it issued is still    */
                              /*   waited for, with the normal one-second bound); the solve returns          */
                              /*   LS_ECUDA.  value = 0 turns it off                                         */
  LS_INJECT_BOUNDS_PROBE = 5  /* plan: value != 0: in the debug build (ls_debug_bounds) the plain first     */
                              /*   pass's slot check excludes the launch's last view, which then fails the   */
                              /*   check (site 0x601) and is skipped; the normal build ignores it           */
};
int ls_debug_inject(ls_plan* plan, int kind, long long value);

/* Index checks of the debug build (the paper has no counterpart).  libls_debug.so is the library
 * compiled with LS_DEBUG_BOUNDS: its hot kernels (the five FFT passes, the bulk-staged first pass,
 * the z passes and the BiCGStab update) test every checked global or shared-memory index against
 * the extents of its array; a failing check records a site code (kernel << 8 | access) and the
 * access is skipped, so a wrong index never faults.  *site (host, may be NULL) receives the first
 * recorded code over the library's translation units (0: none); clear = 1 resets the records.
 * Returns 1 in the debug build, 0 in the normal one (*site = 0; nothing is checked), LS_ECUDA if
 * a record cannot be read.  Reads device memory: call it after the checked work has completed. */
int ls_debug_bounds(unsigned* site, int clear);

/* Measured FP32 throughput of the current device, for the FP32-pipe roofline of the FFT passes (no
 * counterpart in the paper): out[0] scalar FFMA, out[1] scalar FMUL, out[2] packed add.f32x2, each in
 * float lane operations per second (a packed add counts two), from kernels of known operation counts
 * (eight independent dependency chains per thread, eight 256-thread blocks per SM) timed with CUDA
 * events.  out: host array of 3 doubles.  Synchronous on cuda_stream. */
int ls_fp32_peak(double* out, void* cuda_stream);

/* ---------------------------------------------------------------- misc */

const char* ls_status_string(int status);
const char* ls_last_error(void);
/* Device memory (bytes) a plan for this grid and n_views views needs at steady state. */
size_t ls_workspace_bytes(const ls_grid* grid, int n_views);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* LS_H */
