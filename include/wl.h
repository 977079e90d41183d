/*
 * wl.h -- C ABI of the B300 (sm_103a) BDIM incompressible-flow time step.
 *
 * The library advances the velocity/pressure of an incompressible viscous flow
 * around an immersed body on a uniform staggered Cartesian grid (cell size
 * h = 1), following WaterLily (arXiv 2407.16032):
 *   Sec. 2  the momentum equation (F-dot) integrated with an explicit
 *           predictor-corrector (Heun), the boundary-data-immersion (BDIM)
 *           blend (F-dot convolved with the body equation B through the
 *           kernel moments mu0/mu1 of the signed distance), the pressure
 *           projection with a variable-coefficient Poisson equation solved by
 *           geometric multigrid, and a CFL-limited time step;
 *   Sec. 3  the problem statement Simulation(dims, U, L; nu, body) with the
 *           body given by a distance function plus a motion map (AutoBody),
 *           and the pressure-gradient update u[I,i] -= c[I,i](p[I]-p[I-d(i)]);
 *   Sec. 4  the boundary conditions: slip walls, inflow, convective outlet,
 *           periodic directions.
 *
 * Conventions for every entry point:
 *   - Returns a wl_status; nothing throws or aborts across the ABI.
 *     On error, wl_last_error(sim) describes it and the simulation state stays
 *     defined (the last completed step's fields are kept).
 *   - Field layout: component-major, x fastest. A velocity field of an
 *     ndim-dimensional grid n[0] x n[1] (x n[2]) is ndim consecutive arrays of
 *     n[0]*n[1]*n[2] values; value (a, i, j, k) sits at
 *     a*N + i + n[0]*(j + n[1]*k), N = n[0]*n[1]*n[2].  Component a lives on
 *     the lower a-face of cell (i,j,k), i.e. at (i+1/2, j+1/2, k+1/2) - e_a/2.
 *     The exit plane (convective outlet, upper x face) holds n[1]*n[2] values
 *     of u_x at x = n[0], index j + n[1]*k.
 *   - Element type: float for WL_F32, double for WL_F64 (velocity, coefficient
 *     and body arrays); pressure and scalars are always double on the host side.
 *   - Pointers: any argument documented "host or device" may point to host
 *     memory (pageable or pinned) or to device memory of the sim's device;
 *     the library copies with cudaMemcpyAsync(cudaMemcpyDefault) on the sim's
 *     stream and synchronises that stream before returning.  Caller keeps
 *     ownership of every pointer it passes; the sim owns what it allocates.
 *   - All device work is enqueued on cfg.stream.  One sim must not be used by
 *     two host threads at once.
 */
#ifndef WL_H
#define WL_H

#include <stddef.h>

#if defined(__GNUC__)
#define WL_API __attribute__((visibility("default")))
#else
#define WL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wl_sim wl_sim;

typedef enum {
    WL_OK = 0,
    WL_ERR_ARG = 1,            /* invalid argument or configuration */
    WL_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    WL_ERR_ALLOC = 3,          /* device allocation failed */
    WL_ERR_NOT_CONVERGED = 4,  /* Poisson solve hit itmax before tol */
    WL_ERR_NONFINITE = 5,      /* NaN/Inf appeared in the solution */
    WL_ERR_UNSTABLE = 6,       /* CFL time step fell below dt_min */
    WL_ERR_STATE = 7           /* call not valid in the current state */
} wl_status;

typedef enum { WL_F32 = 0, WL_F64 = 1 } wl_precision;

/* USER_FACE_FIELDS: a body of any shape and motion whose distance, normal and
 * velocity the caller samples on the grid (wl_set_body_fields); the other
 * wl_body members are ignored for it. */
typedef enum {
    WL_BODY_NONE = 0,
    WL_BODY_SPHERE = 1,
    WL_BODY_ELLIPSE = 2,
    WL_BODY_CYLINDER = 3,
    WL_BODY_USER_FACE_FIELDS = 4
} wl_body_kind;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` (256-byte aligned) or
 * NULL; free releases it. NULL alloc => cudaMalloc/cudaFree. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes);
    void (*free)(void *ctx, void *ptr);
} wl_allocator;

/* Problem statement (Sec. 3 Simulation; Sec. 4 boundary conditions). */
typedef struct {
    int ndim;              /* 2 or 3 */
    int n[3];              /* cells per axis (n[2] ignored when ndim == 2) */
    int periodic[3];       /* nonzero: periodic axis */
    int exit_hi_x;         /* nonzero: convective outlet on the upper x face */
    double U[3];           /* free stream: normal velocity of non-periodic boundary faces */
    double nu;             /* kinematic viscosity (grid units) */
    double eps;            /* BDIM kernel half-width (1 = one cell) */
    int precision;         /* wl_precision */
    double cfl;            /* CFL number for the adaptive time step (1) */
    double dt_max;         /* upper bound of the adaptive time step (1) */
    double dt_init;        /* first time step (0.25) */
    double dt_min;         /* below this the step reports WL_ERR_UNSTABLE (1e-6) */
    double tol;            /* relative L2 residual of each Poisson solve (1e-6) */
    int itmax;             /* max multigrid V-cycles per solve (32) */
    int smooth_iters;      /* PCG smoothing iterations per level (4) */
    void *stream;          /* cudaStream_t; NULL = legacy default stream */
    wl_allocator allocator;
} wl_config;

/* Analytic immersed body (Sec. 3 AutoBody: signed distance + motion map).
 * SPHERE is a circle in 2D. CYLINDER (3D) is a circular cylinder of the given
 * radius with its axis along z through (centre[0], centre[1]) (the moving
 * cylinder benchmark of Sec. 4, spanwise periodic). The centre heaves along heave_axis as
 * centre + heave_amp sin(omega t + phase); ELLIPSE (2D) has semi-axes semi[0]
 * (chord/2, along x at zero pitch) and semi[1] (thickness/2) and pitches about
 * its centre by pitch_amp sin(omega t + phase + pi/2). Signed distance d > 0 in
 * the fluid; normal = grad d (into the fluid); V = rigid-body velocity. */
typedef struct {
    int kind;              /* wl_body_kind */
    double centre[3];
    double radius;
    double semi[2];
    double heave_amp, pitch_amp, omega, phase;
    int heave_axis;
} wl_body;

typedef struct {
    int vcycles;           /* V-cycles used */
    double rel_resid;      /* final |b - A p|_2 / |b|_2 over active rows */
    double bnorm;          /* |b|_2 of the mean-free right-hand side */
    double rel_initial;    /* relative residual of the initial guess (after the learned guess, if used) */
} wl_solve_stats;

typedef struct {
    wl_solve_stats proj[2];  /* predictor and corrector projections */
    double dt;               /* time step taken */
    double t;                /* time after the step */
    double dt_next;          /* CFL time step for the next step */
} wl_step_stats;

/* Fill *cfg with defaults for an ndim grid of n cells (free stream 0, slip
 * walls, FP32, tol 1e-6, itmax 32, 4 smoothing iterations, eps 1, cfl 1). */
WL_API void wl_config_default(wl_config *cfg, int ndim, const int *n);

/* Create a simulation (Sec. 3 Simulation(dims, U, L; nu, body)).
 * Allocates all device state on the current device, measures the body at
 * t = 0, sets u = 0 with U on the inflow/wall faces and the exit plane, p = 0.
 * body may be NULL (no body). Errors: WL_ERR_ARG (bad sizes or 2^31 cells or more, ndim, eps <= 0,
 * nu < 0, ellipse in 3D, exit without non-periodic x), WL_ERR_ALLOC, WL_ERR_CUDA. */
WL_API int wl_sim_create(const wl_config *cfg, const wl_body *body, wl_sim **out);

/* Free everything the sim allocated. NULL is accepted. */
WL_API int wl_sim_destroy(wl_sim *sim);

/* Copy a velocity field in (host or device; cfg.precision element type;
 * layout above). ue may be NULL when there is no exit plane. The lower
 * boundary faces of non-periodic axes are overwritten with U. */
WL_API int wl_set_velocity(wl_sim *sim, const void *u, const void *ue);

/* Copy the velocity field (and exit plane, if ue != NULL) out (host or device). */
WL_API int wl_get_velocity(wl_sim *sim, void *u, void *ue);

/* Pressure (doubles, one per cell, host or device). get returns the pressure of
 * the last projection with zero mean over active cells and 0 in cells whose
 * faces are all solid; set gives the warm start of the next solve. */
WL_API int wl_get_pressure(wl_sim *sim, double *p);
WL_API int wl_set_pressure(wl_sim *sim, const double *p);

/* Simulation time and the time step the next wl_mom_step will use. */
WL_API int wl_set_time(wl_sim *sim, double t, double dt_next);
WL_API int wl_get_time(wl_sim *sim, double *t, double *dt_next);

/* One Heun predictor-corrector step with two projections (Sec. 2):
 *   u0 = u; u* = P_1[ B(u0 + dt R(u0)) ];  u = P_1/2[ (u* + B(u0 + dt R(u*)))/2 ]
 * where R is the convection-diffusion flux, B the BDIM blend (with the body
 * measured at t + dt), and P_w the projection with weight w. dt_fixed > 0 uses
 * that step; otherwise the CFL step computed after the previous step.
 * Errors: WL_ERR_NOT_CONVERGED (state advanced, residual above tol),
 * WL_ERR_NONFINITE, WL_ERR_UNSTABLE (state kept), WL_ERR_CUDA. stats may be NULL. */
WL_API int wl_mom_step(wl_sim *sim, double dt_fixed, wl_step_stats *stats);

/* Project the current velocity: solve A P = div(u)/(w dt) and set
 * u -= w dt c grad P (Sec. 3 listing), P warm-started from the last solve. */
WL_API int wl_project(wl_sim *sim, double w, double dt, wl_solve_stats *stats);

/* Solve A p = b - mean(b) with the sim's current coefficients.
 * b: cfg.precision element type, host or device; p: doubles, host or device,
 * warm start in / solution out (zero mean over active cells). */
WL_API int wl_poisson_solve(wl_sim *sim, const void *b, double *p, wl_solve_stats *stats);

/* Convection-diffusion right-hand side r = R(u) (Sec. 2 F-dot without the
 * pressure term) of a given field u (+ exit plane ue, may be NULL), into r.
 * All three host or device, cfg.precision element type. r is 0 on the lower
 * boundary faces of non-periodic axes. Uses the sim's scratch buffers. */
WL_API int wl_conv_diff(wl_sim *sim, const void *u, const void *ue, void *r);

/* Pressure force on the body, F = -sum_I p_I n(x_I) K_eps(d(x_I)) over cell
 * centres (the BDIM kernel-weighted surface integral), p the pressure with its
 * mean over active cells removed (as wl_get_pressure reports it), at the time
 * the body was last measured. F: 3 doubles (host); 0 without a body. */
WL_API int wl_forces(wl_sim *sim, double *F);

/* Viscous force on the body (the paper prints no force formula; Sec. 5 reports
 * drag): the traction nu (grad u + grad u^T) . n of the viscous stress, spread
 * over the kernel band like the pressure force,
 *   F_a = nu sum_I K_eps(d(x_I)) sum_b S_ab(x_I) n_b(x_I),  S = grad u + grad u^T,
 * with the gradient at the cell centre from the face samples (d_a u_a =
 * u_a[I+e_a] - u_a[I]; d_b u_a the mean of the two central differences of the
 * faces I and I+e_a, b != a). n = grad d points into the fluid, so the total
 * force on the body is wl_forces + wl_forces_viscous. Uses the current velocity
 * and the body at the time it was last measured. F: 3 doubles (host); 0 without
 * a body. */
WL_API int wl_forces_viscous(wl_sim *sim, double *F);

/* Measure the body at time t onto the faces (mu0, mu1 n, V) and rebuild the
 * multigrid coefficients (Sec. 2 / Sec. 3 measure of AutoBody). For a
 * WL_BODY_USER_FACE_FIELDS body the fields stay as last set and only the time
 * they stand for moves to t. */
WL_API int wl_body_update(wl_sim *sim, double t);

/* Set the body of a WL_BODY_USER_FACE_FIELDS sim from samples of its signed
 * distance function and motion map (Sec. 3 AutoBody: the caller evaluates the
 * distance, its gradient and the body velocity; Sec. 2 forms the kernel
 * moments). All arrays are in cfg.precision, host or device, x fastest
 * (layout of wl_set_velocity), nc = n0 n1 (n2) cells; face a of cell I sits at
 * I + 1/2 - e_a/2 (unit cells), the centre of cell I at I + 1/2:
 *   d_face: ndim arrays, signed distance at face a (> 0 in the fluid);
 *   n_face: ndim*ndim arrays, array a*ndim + b = component b of the unit normal
 *           (grad d, into the fluid) at face a;
 *   V_face: ndim arrays, component a of the body velocity at face a;
 *   d_cell: 1 array, signed distance at the cell centres (forces);
 *   n_cell: ndim arrays, unit normal at the cell centres (forces).
 * The library copies them, forms mu0(d) and mu1(d) n on every face in double
 * precision (rounded once to cfg.precision), zeroes the lower boundary faces
 * of non-periodic axes, and rebuilds every multigrid level's coefficients,
 * 1/D, tile flags and coarsest operator. The fields hold until the next call
 * (steps do not re-measure such a body: set the fields for t + dt before a
 * step to move it); until the first call the grid is all fluid. Drops a held
 * window. Errors: WL_ERR_ARG (another body kind, a NULL array), WL_ERR_CUDA. */
WL_API int wl_set_body_fields(wl_sim *sim, const void *d_face, const void *n_face, const void *V_face,
                              const void *d_cell, const void *n_cell);

/* Tangent of a WL_BODY_USER_FACE_FIELDS body's face velocity along one scalar
 * parameter theta (layout of V_face; cfg.precision, host or device), for a body
 * whose geometry does not depend on theta (e.g. the spin rate of a circular
 * cylinder). wl_window_backward's dparams[0] is then dJ/dtheta through the
 * BDIM blend's body velocity (dparams[1] = 0). NULL clears it (dparams = 0).
 * Errors: WL_ERR_ARG (another body kind), WL_ERR_CUDA. */
WL_API int wl_set_body_velocity_tangent(wl_sim *sim, const void *dV_face);

/* Copy the measured face fields out (host or device, cfg.precision type):
 * c = Poisson coefficients (mu0 with non-periodic lower boundary faces zeroed,
 * ndim arrays), mu1n = mu1 * n_b on face a at (a*3+b) (9 arrays, b >= ndim
 * zero), V = body velocity (ndim arrays). Any may be NULL. */
WL_API int wl_get_body_fields(wl_sim *sim, void *c, void *mu1n, void *V);

/* Kinetic energy (mean over cells of |u|^2/2, u at cell centres), mean squared
 * vorticity over cell edges, and max |div u| over active cells. Host doubles. */
WL_API int wl_diagnostics(wl_sim *sim, double *ke, double *enstrophy, double *max_div);

/* Number of multigrid levels and the kernel launch counter (kernels launched
 * by this sim since creation). */
WL_API int wl_info(wl_sim *sim, int *levels, long long *launches);

/* Per-kernel timing mode. on != 0: every kernel of the following calls is
 * bracketed by CUDA events on the sim's stream (the multigrid V-cycle then runs
 * as direct launches instead of its CUDA graph) and times are accumulated per
 * kernel and multigrid level; on == 0 stops it. Enabling clears the totals. */
WL_API int wl_profile(wl_sim *sim, int on);

/* Text report of the accumulated timing, one line per kernel and level:
 * "name level launches total_ms cells_per_launch". Writes at most len bytes
 * (NUL-terminated) into buf; *needed (may be NULL) receives the full size. */
WL_API int wl_profile_report(wl_sim *sim, char *buf, size_t len, size_t *needed);

/* Learned Poisson initial guess (no counterpart in the paper; its data-driven
 * multigrid reference, Sec. 3, is the precedent). A bias-free ReLU 3D
 * convolutional network with 3x3x3 kernels and channels 1 -> 16 -> 16 -> 1 runs
 * on multigrid level `level` (1/2^level of each axis): it maps the restricted
 * residual of the warm start to a coarse pressure correction, which is added to
 * the pressure by injection before the V-cycles; the V-cycles then converge to
 * the same tolerance (the guess only changes where they start, never when
 * they stop).
 * Convolutions run on BF16 tensor cores with FP32 accumulation (tcgen05 MMAs
 * into tensor memory for the forward and data-gradient convolutions, mma.sync
 * for the weight gradient); weights are kept in FP32 (Adam) and copied to BF16.
 * A tensor-core wait that times out ends the call with WL_ERR_CUDA.
 *   wl_guess_setup: allocate the network and room for `capacity` samples.
 *   wl_guess_mode: collect != 0 records (restricted residual, coarse mean of
 *     the converged-minus-initial pressure) of every converged projection;
 *     use != 0 applies the trained network to every projection.
 *   wl_guess_train: `iters` Adam steps of `batch` samples each on the GPU;
 *     loss = sum (y - t)^2 / sum t^2; first and last losses returned.
 *   wl_guess_weights: set (in) and/or get (out) the FP32 weights,
 *     3 x 27 x 16 x 16 floats [layer][tap z,y,x][in][out] (host or device).
 *   wl_guess_info: level, number of samples held, output gain. */
WL_API int wl_guess_setup(wl_sim *sim, int level, int capacity);
WL_API int wl_guess_mode(wl_sim *sim, int collect, int use);
WL_API int wl_guess_train(wl_sim *sim, int iters, double lr, int batch, unsigned seed, double *loss_first,
                          double *loss_last);
WL_API int wl_guess_weights(wl_sim *sim, const float *in, float *out);
WL_API int wl_guess_info(wl_sim *sim, int *level, int *samples, double *gain);

/* Learned temporal guess (no counterpart in the paper): a 1x1x1 convolution
 * over the pressure history of each projection stage (predictor, corrector),
 *   guess = H1 + w1 (H1 - H2) + w2 (Ho - H1),
 * H1, H2 the stage's last two converged pressures, Ho the other stage's latest
 * (w = (0, 1) is the plain warm start from the previous projection). It
 * replaces the warm start of each wl_mom_step projection once two steps of
 * history exist; the V-cycles then converge to the same tolerance (the guess
 * only changes where they start). When both learned guesses are on,
 * this one is applied first and the network's coarse correction after it.
 *   wl_tguess_mode: collect != 0 gathers, at every converged projection, the
 *     normal equations of the weights' least-squares fit in the residual norm
 *     |A (P - guess)| (entering collection clears them); use != 0 applies
 *     the weights. The history restarts after wl_set_velocity/_pressure.
 *   wl_tguess_fit: fits (w1, w2) per stage from the gathered equations; w:
 *     4 doubles (predictor w1, w2, corrector w1, w2), ratio: 2 doubles, the
 *     fitted guess's residual norm over the plain warm start's on the
 *     collected projections (either may be NULL).
 *   wl_tguess_weights: set (in) and / or get (out) the 4 weights (host). */
WL_API int wl_tguess_mode(wl_sim *sim, int collect, int use);
WL_API int wl_tguess_fit(wl_sim *sim, double *w, double *ratio);
WL_API int wl_tguess_weights(wl_sim *sim, const double *in, double *out);

/* One forward and backward pass of the guess network on a single sample (for
 * checking the kernels): grid ndim, n[3]; weights w (3 x 27 x 16 x 16 floats);
 * input x and target t (n[0]*n[1]*n[2] floats, t may be NULL for forward
 * only); outputs y (forward result), dw (gradient of the loss w.r.t. w) and
 * the loss. All host or device pointers. Allocates its own device buffers.
 * Grids of more than 134217727 cells (2^31 / 16: the kernels index voxel x
 * channel in 32-bit integers) give WL_ERR_ARG before any device work; the same
 * bound applies to the level chosen by wl_guess_setup. */
WL_API int wl_net_eval(int ndim, const int *n, const float *w, const float *x, const float *t, float *y, float *dw,
                       double *loss);

/* Adjoint of one time step (no counterpart in the paper, which differentiates
 * the solver in forward mode with dual numbers, Sec. 3 / Sec. 6.1): the
 * vector-Jacobian product of wl_mom_step with the fixed step dt from the start
 * state (u0, ue0) at time t, the body measured at t + dt as the step does.
 * Given the cotangents lu (velocity), le (exit plane, may be NULL) and lP
 * (reported pressure, nc doubles, may be NULL) of the step's outputs, returns
 * ub, ueb = J^T (lu, le, lP) for (u0, ue0). The Jacobian is taken with the
 * flux limiter's branches frozen at the evaluation point. Transposes: the
 * convection-diffusion flux (scattered), the BDIM blend (gathered), the exit
 * condition, and each projection through one Poisson solve on div(c lam) with
 * the same symmetric multigrid, converged to relative residual `tol` (the
 * forward projection inside is solved to `tol` too).
 *   u0, lu, ub: ndim arrays of nc (cfg.precision type); ue0, le, ueb: the exit
 *   plane (ignored / may be NULL without an exit); P0: warm start of the
 *   forward projection (nc doubles, may be NULL = 0). All host or device.
 * The sim's velocity, pressure, time and body are unchanged on return.
 * stats (may be NULL): the two adjoint solves (predictor, corrector).
 * Errors: WL_ERR_ARG, WL_ERR_NOT_CONVERGED, WL_ERR_NONFINITE, WL_ERR_CUDA. */
WL_API int wl_step_vjp(wl_sim *sim, double t, double dt, const void *u0, const void *ue0, const double *P0,
                       const void *lu, const void *le, const double *lP, double tol, void *ub, void *ueb,
                       wl_solve_stats *stats);

/* Derivative of the pressure force (wl_forces) component `axis` with respect
 * to the reported pressure, times `scale`: g[I] = -scale n_axis(x_I)
 * K_eps(d(x_I)) on active cells (0 elsewhere), body at its last measured time.
 * g: nc doubles, host or device. */
WL_API int wl_force_dp(wl_sim *sim, int axis, double scale, double *g);

/* Gradient over a window of time steps, with checkpointed recomputation (no
 * counterpart in the paper; its forward-mode dual numbers, Sec. 3 / Sec. 6.1,
 * are replaced by the step's hand-written adjoint, wl_step_vjp). Objective:
 *   J = sum_{n=1..nsteps} w . F_n  (+ <lu, u_N> + <le, ue_N> in the backward call)
 * with F_n the pressure force of wl_forces after step n (mean thrust of a
 * flapping foil: w = (-1/nsteps, 0, 0)).
 *   wl_window_forward: runs nsteps steps from the current state with the time
 *     steps dts (nsteps doubles; NULL = the adaptive CFL steps, which are then
 *     held fixed for the gradient), storing a checkpoint of the state every
 *     ckpt_every steps on the device (ceil(nsteps/ckpt_every) + ckpt_every + 1
 *     states of velocity, exit plane and pressure). Returns J (may be NULL) and
 *     the steps taken (dts_out, may be NULL). w: 3 doubles (NULL = 0).
 *   wl_window_backward: the reverse sweep. Each segment is recomputed from its
 *     checkpoint, then the steps are pulled back with wl_step_vjp's kernels,
 *     the adjoint Poisson solves converged to `tol`. Inputs: gJ (the cotangent
 *     of J), lu / le (cotangents of the final velocity and exit plane, may be
 *     NULL = 0). Outputs (each may be NULL): du0, due0 (gradient with respect
 *     to the window's start velocity and exit plane, layout of wl_set_velocity)
 *     and dparams (host, 2 doubles): (dJ/d heave_amp, dJ/d pitch_amp) of an
 *     analytic body, through the measured face fields, the Poisson
 *     coefficients and the force's own dependence on the body; (dJ/d theta, 0)
 *     of a sampled body along its velocity tangent. The sim is left in the state
 *     after the window. Errors: WL_ERR_STATE (no forward window held),
 *     WL_ERR_NONFINITE, WL_ERR_ARG, WL_ERR_CUDA; a forward step that fails
 *     returns its status from wl_window_forward. */
WL_API int wl_window_forward(wl_sim *sim, int nsteps, int ckpt_every, const double *dts, const double *w, double *J,
                             double *dts_out);
/* wl_window_forward with per-step weights and an optional viscous part:
 * J = sum_n step_w[n] w . F_n (step_w: nsteps doubles, host; NULL = all 1),
 * e.g. the force at the final step alone, with F_n = wl_forces, plus
 * wl_forces_viscous when viscous != 0 (the total force on the body).
 * wl_window_backward then pulls back this J; the viscous force is linear in
 * the velocity, so its part adds a fixed field to each weighted step's
 * velocity cotangent. */
WL_API int wl_window_forward_weighted(wl_sim *sim, int nsteps, int ckpt_every, const double *dts, const double *w,
                                      const double *step_w, int viscous, double *J, double *dts_out);
WL_API int wl_window_backward(wl_sim *sim, double gJ, const void *lu, const void *le, double tol, void *du0,
                              void *due0, double *dparams);

/* Checkpoint and resume. wl_state_size gives the bytes of the sim's state;
 * wl_get_state writes it to buf (host or device, at least that many bytes):
 * a header (format version, ndim, n, precision, body kind), the time, the
 * next CFL time step and the time the body was last measured, then the
 * velocity (ndim arrays), the exit plane and the pressure pair (high and low
 * parts, the warm start of the next solve), in cfg.precision. wl_set_state
 * loads it into a sim created with the same configuration and body: a body
 * is measured again at its saved time, so the steps that follow equal, bit
 * for bit, those of the sim the state was taken from. Not included: a held
 * window, the learned guesses' fitted state (resume with them off, or fit
 * them again), a WL_BODY_USER_FACE_FIELDS body's samples (set the same
 * fields on the resumed sim, before or after wl_set_state), and the
 * coarsest-level setting of wl_set_coarse_dense_max (set it on the resumed
 * sim as on the original). Errors: WL_ERR_ARG (NULL buffer, too small, a state of another
 * grid, precision or body kind), WL_ERR_CUDA. */
WL_API int wl_state_size(wl_sim *sim, size_t *bytes);
WL_API int wl_get_state(wl_sim *sim, void *buf, size_t bytes);
WL_API int wl_set_state(wl_sim *sim, const void *buf, size_t bytes);

/* Adjoint Poisson solves of the last wl_window_backward (two per step):
 * counts[0] solves, counts[1] solves that stopped above tol (the sweep goes on
 * with them: their steps' share of the gradient is then less accurate),
 * counts[2] the largest V-cycle count, counts[3] the window step (0-based) of
 * the largest final relative residual, *max_rel that residual. Either
 * pointer may be NULL. */
WL_API int wl_window_stats(wl_sim *sim, int *counts, double *max_rel);

/* Replace the body's parameters (same kind; e.g. new heave / pitch amplitudes)
 * and re-measure it at the time it was last measured. Drops a held window. */
WL_API int wl_set_body(wl_sim *sim, const wl_body *body);

/* How the coarsest level of the multigrid V-cycle (Sec. 2, geometric
 * multigrid; Sec. 4.2, the pressure solver) is solved. A coarsest level of at
 * most max_cells cells is solved by a dense FP64 solution operator (the
 * inverse of the level's operator bordered by the mean constraint, built on
 * the device by one PCG solve per column, again after every measure of a
 * moving or sampled body) and a matrix-vector product; a larger one by
 * Jacobi-PCG in FP64 on one thread block, to 1e-12 relative. Both give the
 * level's exact mean-free solution up to rounding. The hierarchy halves every
 * axis while all are even and all halves are at least 4, so a grid such as
 * 9L x 6L x 2L keeps a coarsest level of 864 cells, where the one-block PCG
 * can take most of a step; max_cells = 1024 moves it onto the dense
 * operator. It holds 5 n^2 doubles of device memory, 40 MiB at most: the
 * operator and its build's scratch. The build costs about n one-block solves,
 * once per measure of a moving body.
 *   max_cells: 0 .. 1024 (256 when a sim is created; 0 = always PCG).
 * Drops a held window. Errors: WL_ERR_ARG (out of range, NULL sim),
 * WL_ERR_CUDA. */
WL_API int wl_set_coarse_dense_max(wl_sim *sim, int max_cells);

/* Largest grid (cells) wl_coarse_solve_static accepts: its working memory is
 * a fixed device array of 5 * WL_STATIC_MAX_CELLS + 8 doubles (~640 KiB) that
 * every GPU loading this library holds until the process exits. */
#define WL_STATIC_MAX_CELLS 16384

/* Poisson solve that allocates no device memory (no counterpart in the paper:
 * an addition for callers that cannot call cudaMalloc when they need the
 * solve: an application whose device memory is entirely held by its own pool
 * or budget, so that a library allocation would fail or break the budget, and
 * a time-critical loop that must not call cudaMalloc because the call can
 * synchronise the device and stall the work on every stream). Solves, on one
 * thread block (up to 1024 threads) in double precision,
 * A x = r - mean(r) with the operator and Jacobi-preconditioned CG of the
 * library's coarsest multigrid level (the mean is over rows with a nonzero
 * diagonal; x is returned mean-free over those rows and 0 elsewhere).
 *   ndim, n[3], periodic[3]: the grid (n[2] ignored in 2D);
 *   precision: element type of c, r, x (WL_F32 float, WL_F64 double);
 *   c[a]: device array of the lower a-face coefficients of every cell (the
 *         layout of include/wl.h fields); the upper faces of non-periodic axes
 *         are taken as 0, and the caller gives 0 on their lower faces;
 *   r, x: device arrays (x is written, r is read; they must not alias);
 *   maxit, rtol: CG iteration limit and relative residual target;
 *   stream: cudaStream_t (NULL = legacy default stream);
 *   rel_resid: if not NULL, receives the final relative residual (the call
 *         then synchronises the stream); if NULL the call only enqueues.
 * The working memory is one file-scope device array shared by every call: it
 * keeps the last call's contents and the solve re-initialises what it reads;
 * calls that may overlap on the GPU (on different streams or host threads)
 * race on it and must be serialised by the caller. The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 * Errors: WL_ERR_ARG for bad arguments or n[0]*n[1]*n[2] > WL_STATIC_MAX_CELLS,
 * WL_ERR_CUDA if the address lookup or the launch fails. */
WL_API int wl_coarse_solve_static(int ndim, const int *n, const int *periodic, int precision,
                                  const void *const *c, const void *r, void *x, int maxit, double rtol,
                                  void *stream, double *rel_resid);

WL_API const char *wl_last_error(const wl_sim *sim);
WL_API const char *wl_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
