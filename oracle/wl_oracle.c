/*
 * wl_oracle.c -- plain, slow FP64 CPU oracle of one BDIM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the bench's CPU-baseline
 * leg do.  It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (WaterLily, arXiv 2407.16032):
 *   Sec. 2  -- momentum equation F-dot (u_i' = -p_,i - (u_i u_j)_,j + nu u_i,jj),
 *              body equation B (u_i = V_i), convolved through the BDIM kernel
 *              of half-width eps using the signed distance d and normal n.
 *   Sec. 2  -- finite volume, uniform Cartesian staggered grid (h = 1), central
 *              differences for pressure and diffusion, flux-limited QUICK for
 *              convection, explicit predictor-corrector (Heun) in time, pressure
 *              projection with a variable-coefficient Poisson equation solved by
 *              geometric multigrid, CFL-adapted time step.
 *   Sec. 3  -- pressure-gradient update u[I,i] -= c[I,i]*(p[I]-p[I-d(i)]),
 *              with c the Poisson coefficients; velocity component i on the
 *              lower i-face of cell I.
 *   Sec. 4.2 -- multigrid uses a preconditioned-conjugate-gradient smoother.
 *
 * Where the paper is silent the reading taken is written next to the code
 * (grid coordinates, the QUICK variant and limiter, boundary treatment, the
 * kernel moments, the exit condition, multigrid details, CFL formula).
 *
 * Layout: every field is component-major, x fastest: u[a*nc + i + n0*(j + n1*k)].
 *
 * Threads: the per-cell loops carry OpenMP pragmas (compiled with -fopenmp;
 * without it they are ignored). Every cell's value is computed by the same
 * expression whatever thread runs it, and every sum over cells uses a fixed
 * blocked order (fixed_sum), so results are bitwise identical for any number
 * of threads. The adjoint routines, whose loops scatter, stay serial.
 * 2D uses n[2] = 1 and ndim = 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* Number of OpenMP threads of the per-cell loops (1 without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int ndim;
    int n[3];
    int periodic[3];
    int exit_hi_x;       /* convective outlet on the upper x face */
    double U[3];         /* free-stream velocity (boundary normal values) */
    double nu;
    double eps;          /* BDIM kernel half-width */
} orc_grid;

typedef struct {
    int kind;            /* 0 none, 1 sphere (circle in 2D), 2 ellipse (2D) */
    double centre[3];
    double radius;
    double semi[2];      /* ellipse semi-axes along chord and thickness */
    double heave_amp, pitch_amp, omega, phase;
    int heave_axis;
} orc_body;

typedef struct {
    double tol;          /* relative L2 residual target */
    int itmax;           /* max V-cycles */
    int smooth_iters;    /* PCG iterations per level (post-smoothing) */
} orc_solver;

typedef struct {
    int vcycles;
    double rel_resid;
    double bnorm;
} orc_stats;

static inline size_t ncell(const orc_grid *g) { return (size_t)g->n[0] * g->n[1] * g->n[2]; }
static inline size_t lin(const orc_grid *g, int i, int j, int k) {
    return (size_t)i + (size_t)g->n[0] * ((size_t)j + (size_t)g->n[1] * (size_t)k);
}

/* ------------------------------------------------------------------------ */
/* Velocity samples with boundary treatment.                                 */
/* Reading: periodic axes wrap; on a non-periodic axis the tangential        */
/* components are extended by zero gradient (index clamped to the interior), */
/* and the normal component u_a has faces 0..N_a, where face N_a is the upper */
/* boundary face whose value is U_a (slip/inflow) or the stored exit plane.  */
/* Indices beyond are clamped to those end faces (zero-gradient extension).  */
/* ------------------------------------------------------------------------ */
static double su(const orc_grid *g, const double *u, const double *ue, int a, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    int upper = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int N = g->n[ax];
        if (ax >= g->ndim) { idx[ax] = 0; continue; }
        if (g->periodic[ax]) {
            idx[ax] = ((idx[ax] % N) + N) % N;
        } else if (ax == a) {
            if (idx[ax] < 0) idx[ax] = 0;
            if (idx[ax] >= N) { idx[ax] = N; upper = 1; }
        } else {
            if (idx[ax] < 0) idx[ax] = 0;
            if (idx[ax] > N - 1) idx[ax] = N - 1;
        }
    }
    if (upper) {
        if (a == 0 && g->exit_hi_x) return ue[(size_t)idx[1] + (size_t)g->n[1] * idx[2]];
        return g->U[a];
    }
    return u[(size_t)a * ncell(g) + lin(g, idx[0], idx[1], idx[2])];
}

/* Sample of a stored face array with every axis clamped / wrapped to the stored
 * range (used for the BDIM gradient term and the body velocity). */
static double sc(const orc_grid *g, const double *f, int a, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    for (int ax = 0; ax < 3; ++ax) {
        int N = g->n[ax];
        if (ax >= g->ndim) { idx[ax] = 0; continue; }
        if (g->periodic[ax]) idx[ax] = ((idx[ax] % N) + N) % N;
        else { if (idx[ax] < 0) idx[ax] = 0; if (idx[ax] > N - 1) idx[ax] = N - 1; }
    }
    return f[(size_t)a * ncell(g) + lin(g, idx[0], idx[1], idx[2])];
}

/* ------------------------------------------------------------------------ */
/* Flux-limited QUICK face value (Sec. 2: QUICK with a flux limiter).          */
/* Reading: upwind-biased third-order interpolation (5c + 2d - u)/6 limited  */
/* by median(phi, c, median(10c - 9u, c, d)), u/c/d being the far-upstream,  */
/* upstream and downstream samples.                                          */
/* ------------------------------------------------------------------------ */
static double median3(double a, double b, double c)
{
    return fmax(fmin(a, b), fmin(fmax(a, b), c));
}

double orc_quick(double uu, double c, double d)
{
    double phi = (5.0 * c + 2.0 * d - uu) / 6.0;
    return median3(phi, c, median3(10.0 * c - 9.0 * uu, c, d));
}

/* Total (convective + diffusive) flux of u_a through the lower b-face of the
 * u_a control volume of cell I, positive in +b. */
static double face_flux(const orc_grid *g, const double *u, const double *ue, int a, int b, int i, int j, int k)
{
    int db[3] = {0, 0, 0}, da[3] = {0, 0, 0};
    db[b] = 1; da[a] = 1;
    /* advecting velocity: mean of the two u_b samples straddling the face along a */
    double Uf = 0.5 * (su(g, u, ue, b, i, j, k) + su(g, u, ue, b, i - da[0], j - da[1], k - da[2]));
    double sm2 = su(g, u, ue, a, i - 2 * db[0], j - 2 * db[1], k - 2 * db[2]);
    double sm1 = su(g, u, ue, a, i - db[0], j - db[1], k - db[2]);
    double s0 = su(g, u, ue, a, i, j, k);
    double sp1 = su(g, u, ue, a, i + db[0], j + db[1], k + db[2]);
    double phi = (Uf > 0.0) ? orc_quick(sm2, sm1, s0) : orc_quick(sp1, s0, sm1);
    return Uf * phi - g->nu * (s0 - sm1);
}

/* Momentum RHS r = -(u_a u_b)_,b + nu u_a,bb in flux form (Sec. 2, Eq. F-dot
 * without the pressure term). r is zero on the lower boundary face of a
 * non-periodic axis (its value is set by the boundary condition). */
void orc_conv_diff(const orc_grid *g, const double *u, const double *ue, double *r)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    double acc = 0.0;
                    if (!(g->periodic[a] == 0 && I[a] == 0)) {
                        for (int b = 0; b < g->ndim; ++b) {
                            int db[3] = {0, 0, 0};
                            db[b] = 1;
                            acc += face_flux(g, u, ue, a, b, i, j, k)
                                 - face_flux(g, u, ue, a, b, i + db[0], j + db[1], k + db[2]);
                        }
                    }
                    r[(size_t)a * nc + lin(g, i, j, k)] = acc;
                }
}

/* ------------------------------------------------------------------------ */
/* BDIM kernel moments (Sec. 2: thickness eps, signed distance d, normal n). */
/* Kernel K(s) = (1 + cos(pi s/eps))/(2 eps), |s| < eps.  mu0 = integral of  */
/* K over the fluid side, mu1 = first moment of K over the fluid side.       */
/* d > 0 in the fluid, n = grad d points into the fluid (reading).            */
/* ------------------------------------------------------------------------ */
double orc_mu0(double d, double eps)
{
    double r = d / eps;
    if (r <= -1.0) return 0.0;
    if (r >= 1.0) return 1.0;
    return 0.5 * (1.0 + r + sin(OR_PI * r) / OR_PI);
}

double orc_mu1(double d, double eps)
{
    double r = d / eps;
    if (r <= -1.0 || r >= 1.0) return 0.0;
    return eps * (0.25 - 0.25 * r * r - (r * sin(OR_PI * r) + (1.0 + cos(OR_PI * r)) / OR_PI) / (2.0 * OR_PI));
}

double orc_kernel(double d, double eps)
{
    double r = d / eps;
    if (r <= -1.0 || r >= 1.0) return 0.0;
    return (1.0 + cos(OR_PI * r)) / (2.0 * eps);
}

/* Signed distance, unit normal and rigid-body velocity of an analytic body at
 * point x and time t (Sec. 3 AutoBody: distance function + coordinate map). */
void orc_body_eval(const orc_body *B, int ndim, const double *x, double t, double *d, double *nrm, double *V)
{
    double c[3] = {B->centre[0], B->centre[1], B->centre[2]};
    double cdot[3] = {0.0, 0.0, 0.0};
    c[B->heave_axis] += B->heave_amp * sin(B->omega * t + B->phase);
    cdot[B->heave_axis] = B->heave_amp * B->omega * cos(B->omega * t + B->phase);
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    V[0] = cdot[0]; V[1] = cdot[1]; V[2] = cdot[2];
    if (B->kind == 0) { *d = 1e30; return; }
    if (B->kind == 1 || B->kind == 3) {
        /* sphere (circle in 2D); cylinder: the same in the x-y plane, axis along z */
        double r2 = 0.0, rv[3] = {0, 0, 0};
        int na = B->kind == 3 ? 2 : ndim;
        for (int a = 0; a < na; ++a) { rv[a] = x[a] - c[a]; r2 += rv[a] * rv[a]; }
        double rr = sqrt(r2);
        *d = rr - B->radius;
        if (rr > 0.0) for (int a = 0; a < na; ++a) nrm[a] = rv[a] / rr;
        else nrm[0] = 1.0;
        return;
    }
    /* ellipse (2D): body frame x' = Rot(-theta)(x - c); q = |(x'/sa, y'/sb)|;
     * first-order distance d = (q - 1) q / |(x'/sa^2, y'/sb^2)|;
     * normal = direction of grad q (reading); V = cdot + thetadot e_z x (x - c). */
    double th = B->pitch_amp * sin(B->omega * t + B->phase + 0.5 * OR_PI);
    double thd = B->pitch_amp * B->omega * cos(B->omega * t + B->phase + 0.5 * OR_PI);
    double rx = x[0] - c[0], ry = x[1] - c[1];
    double ct = cos(th), st = sin(th);
    double xp = ct * rx + st * ry, yp = -st * rx + ct * ry;
    double sa = B->semi[0], sb = B->semi[1];
    double q = sqrt((xp / sa) * (xp / sa) + (yp / sb) * (yp / sb));
    double gx = xp / (sa * sa), gy = yp / (sb * sb);
    double gn = sqrt(gx * gx + gy * gy);
    if (gn > 0.0) {
        *d = (q - 1.0) * q / gn;
        double nxp = gx / gn, nyp = gy / gn;
        nrm[0] = ct * nxp - st * nyp;
        nrm[1] = st * nxp + ct * nyp;
    } else {
        *d = -sb;
        nrm[0] = 1.0;
    }
    V[0] += -thd * ry;
    V[1] += thd * rx;
}

/* Smallest zeroth moment kept on a face (reading; Sec. 2 is silent on it):
 * below it mu0 is taken as 0, i.e. the face is solid. A cell whose faces sum
 * to a tiny but nonzero coefficient has its pressure fixed only by the
 * rounding of its right-hand side divided by that sum (unbounded as the sum
 * goes to zero, in any precision), and such a cell still counts in the mean
 * over active rows that the pressure is reported against. The cut removes the
 * outermost few percent of the kernel's reach (mu0 ~ pi^2 (1 + r)^3 / 12
 * near r = -1), so no cell sums to less than it without being solid. */
#define OR_MU0_MIN 1e-5
static double mu0_kept(double m) { return m < OR_MU0_MIN ? 0.0 : m; }

/* Measure the body onto every stored face of every component at time t:
 * mu0 (3 x nc), mu1n (9 x nc, index (a*3+b)*nc: mu1 * n_b on face a),
 * V (3 x nc).  Face a of cell I sits at (I + 1/2) - e_a/2. */
void orc_measure(const orc_grid *g, const orc_body *B, double t, double *mu0, double *mu1n, double *V)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    double x[3] = {i + 0.5, j + 0.5, k + 0.5};
                    x[a] -= 0.5;
                    double d, nrm[3], v[3];
                    orc_body_eval(B, g->ndim, x, t, &d, nrm, v);
                    size_t L = lin(g, i, j, k);
                    mu0[(size_t)a * nc + L] = mu0_kept(orc_mu0(d, g->eps));
                    double m1 = orc_mu1(d, g->eps);
                    for (int b = 0; b < 3; ++b) mu1n[(size_t)(a * 3 + b) * nc + L] = (b < g->ndim) ? m1 * nrm[b] : 0.0;
                    V[(size_t)a * nc + L] = v[a];
                }
}

/* Measure a body given by samples instead of a formula (Sec. 3: a body is a
 * distance function plus a map; here the caller evaluates them): on every face
 * a of every cell the signed distance d[a] (> 0 in the fluid), the unit normal
 * n[a*ndim + b] (component b, into the fluid) and the body velocity V[a]
 * (component a). The kernel moments are those of the analytic bodies:
 * mu0 = mu0(d) (cut below OR_MU0_MIN), mu1n = mu1(d) n, V = V (layouts of
 * orc_measure). */
void orc_measure_sampled(const orc_grid *g, const double *d, const double *n, const double *Vin, double *mu0,
                         double *mu1n, double *V)
{
    size_t nc = ncell(g);
    int nd = g->ndim;
    for (int a = 0; a < nd; ++a)
        for (size_t L = 0; L < nc; ++L) {
            double da = d[(size_t)a * nc + L];
            double m1 = orc_mu1(da, g->eps);
            mu0[(size_t)a * nc + L] = mu0_kept(orc_mu0(da, g->eps));
            for (int b = 0; b < 3; ++b)
                mu1n[(size_t)(a * 3 + b) * nc + L] = b < nd ? m1 * n[(size_t)(a * nd + b) * nc + L] : 0.0;
            V[(size_t)a * nc + L] = Vin[(size_t)a * nc + L];
        }
}

/* Pressure force of a sampled body (the reading of orc_forces): F = -sum_I p_I
 * n(x_I) K_eps(d(x_I)) with the distance dc and normal ncen (component b at
 * b*nc) sampled at the cell centres. */
void orc_forces_sampled(const orc_grid *g, const double *dc, const double *ncen, const double *p, double *F)
{
    size_t nc = ncell(g);
    F[0] = F[1] = F[2] = 0.0;
    for (size_t L = 0; L < nc; ++L) {
        double K = orc_kernel(dc[L], g->eps);
        if (K == 0.0) continue;
        double pk = p[L] * K;
        for (int a = 0; a < g->ndim; ++a) F[a] -= pk * ncen[(size_t)a * nc + L];
    }
}

/* Poisson coefficients c_a = mu0 on face a, zero on non-periodic boundary faces
 * (Neumann condition at the domain boundary). */
void orc_coeffs(const orc_grid *g, const double *mu0, double *c)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    size_t L = (size_t)a * nc + lin(g, i, j, k);
                    c[L] = (!g->periodic[a] && I[a] == 0) ? 0.0 : (mu0 ? mu0[L] : 1.0);
                }
}

/* ------------------------------------------------------------------------ */
/* BDIM blend (Sec. 2: F-dot convolved with B):                              */
/*   f = u0 + dt r;  u = V + mu0 (f - V) + mu1 n . grad(f - V)               */
/* with a central difference for the gradient at the face (reading).          */
/* When corrector != 0 the result is averaged with u_star: u = (u* + B(f))/2 */
/* (the Heun corrector). Then lower boundary faces get U_a.                  */
/* ------------------------------------------------------------------------ */
void orc_bdim(const orc_grid *g, const double *u0, const double *r, double dt,
              const double *mu0, const double *mu1n, const double *V,
              const double *ustar, double *out)
{
    size_t nc = ncell(g);
    double *f = (double *)malloc(sizeof(double) * g->ndim * nc);
    for (size_t q = 0; q < (size_t)g->ndim * nc; ++q) f[q] = u0[q] + dt * r[q];
    for (int a = 0; a < g->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    size_t L = (size_t)a * nc + lin(g, i, j, k);
                    double val;
                    if (mu0) {
                        double fv = f[L] - V[L];
                        double grad = 0.0;
                        for (int b = 0; b < g->ndim; ++b) {
                            int db[3] = {0, 0, 0};
                            db[b] = 1;
                            double up = sc(g, f, a, i + db[0], j + db[1], k + db[2]) - sc(g, V, a, i + db[0], j + db[1], k + db[2]);
                            double dn = sc(g, f, a, i - db[0], j - db[1], k - db[2]) - sc(g, V, a, i - db[0], j - db[1], k - db[2]);
                            grad += mu1n[(size_t)(a * 3 + b) * nc + lin(g, i, j, k)] * 0.5 * (up - dn);
                        }
                        val = V[L] + mu0[L] * fv + grad;
                    } else {
                        val = f[L];
                    }
                    if (ustar) val = 0.5 * (ustar[L] + val);
                    if (!g->periodic[a] && I[a] == 0) val = g->U[a];
                    out[L] = val;
                }
    free(f);
}

/* Net volume flux out of the domain through non-periodic boundary faces. */
static double boundary_outflux(const orc_grid *g, const double *u, const double *ue)
{
    double q = 0.0;
    for (int a = 0; a < g->ndim; ++a) {
        if (g->periodic[a]) continue;
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    if (I[a] != 0) continue;
                    int J[3] = {i, j, k};
                    J[a] = g->n[a];
                    q += su(g, u, ue, a, J[0], J[1], J[2]) - su(g, u, ue, a, i, j, k);
                }
    }
    return q;
}

/* Convective exit on the upper x face (Sec. 4: convective outflow boundary).
 * Reading: the exit face value obeys du/dt + Ubar du/dx = 0 with a first-order
 * upwind difference against the last interior u_x face, Ubar = U_x, advanced
 * by the same Heun stages as the interior; afterwards a uniform correction
 * makes the net boundary volume flux exactly zero.
 *   stage 1: ue = ue0 + dt G(ue0, u0)
 *   stage 2: ue = (ue* + ue0 + dt G(ue*, u*))/2,   G(ue, u) = -Ubar (ue - u_x[N-1]) */
void orc_exit_bc(const orc_grid *g, const double *ue0, const double *uG, const double *ueG,
                 double dt, int corrector, const double *ustar_e, double *u_new, double *ue)
{
    if (!g->exit_hi_x) return;
    int n0 = g->n[0], np = g->n[1] * g->n[2];
    double Ubar = g->U[0];
    for (int p = 0; p < np; ++p) {
        int j = p % g->n[1], k = p / g->n[1];
        double last = uG[lin(g, n0 - 1, j, k)];
        double G = -Ubar * (ueG[p] - last);
        double v = ue0[p] + dt * G;
        if (corrector) v = 0.5 * (ustar_e[p] + v);
        ue[p] = v;
    }
    double q = boundary_outflux(g, u_new, ue);
    double corr = -q / (double)np;
    for (int p = 0; p < np; ++p) ue[p] += corr;
}

/* Discrete divergence sum_a (u_a[I+e_a] - u_a[I]). */
void orc_divergence(const orc_grid *g, const double *u, const double *ue, double *div)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double s = 0.0;
                for (int a = 0; a < g->ndim; ++a) {
                    int da[3] = {0, 0, 0};
                    da[a] = 1;
                    s += su(g, u, ue, a, i + da[0], j + da[1], k + da[2]) - su(g, u, ue, a, i, j, k);
                }
                div[lin(g, i, j, k)] = s;
            }
}

/* ------------------------------------------------------------------------ */
/* Variable-coefficient Poisson operator (Sec. 2 / Sec. 3):                  */
/*  (A p)[I] = sum_a c_a[I+e_a](p[I+e_a]-p[I]) - c_a[I](p[I]-p[I-e_a])         */
/* c of the upper boundary face of a non-periodic axis is zero.               */
/* ------------------------------------------------------------------------ */
typedef struct { int ndim; int n[3]; int periodic[3]; double *c; } orc_level;

static size_t lv_nc(const orc_level *L) { return (size_t)L->n[0] * L->n[1] * L->n[2]; }
static size_t lv_lin(const orc_level *L, int i, int j, int k) {
    return (size_t)i + (size_t)L->n[0] * ((size_t)j + (size_t)L->n[1] * (size_t)k);
}
/* coefficient of face a of cell I (I may be one past the end on axis a) */
static double lv_c(const orc_level *L, int a, const int *I)
{
    int J[3] = {I[0], I[1], I[2]};
    if (J[a] == L->n[a]) {
        if (!L->periodic[a]) return 0.0;
        J[a] = 0;
    }
    return L->c[(size_t)a * lv_nc(L) + lv_lin(L, J[0], J[1], J[2])];
}
static double lv_p(const orc_level *L, const double *p, const int *I)
{
    int J[3] = {I[0], I[1], I[2]};
    for (int a = 0; a < L->ndim; ++a) {
        int N = L->n[a];
        if (J[a] < 0) J[a] = L->periodic[a] ? J[a] + N : 0;
        if (J[a] >= N) J[a] = L->periodic[a] ? J[a] - N : N - 1;
    }
    return p[lv_lin(L, J[0], J[1], J[2])];
}

static double lv_apply_row(const orc_level *L, const double *p, int i, int j, int k)
{
    int I[3] = {i, j, k};
    double pI = p[lv_lin(L, i, j, k)];
    double s = 0.0;
    for (int a = 0; a < L->ndim; ++a) {
        int Ip[3] = {i, j, k}, Im[3] = {i, j, k};
        Ip[a] += 1; Im[a] -= 1;
        s += lv_c(L, a, Ip) * (lv_p(L, p, Ip) - pI) - lv_c(L, a, I) * (pI - lv_p(L, p, Im));
    }
    return s;
}

static double lv_diag(const orc_level *L, int i, int j, int k)
{
    int I[3] = {i, j, k};
    double s = 0.0;
    for (int a = 0; a < L->ndim; ++a) {
        int Ip[3] = {i, j, k};
        Ip[a] += 1;
        s -= lv_c(L, a, Ip) + lv_c(L, a, I);
    }
    return s;
}

static void lv_apply(const orc_level *L, const double *p, double *Ap)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < L->n[2]; ++k)
        for (int j = 0; j < L->n[1]; ++j)
            for (int i = 0; i < L->n[0]; ++i) Ap[lv_lin(L, i, j, k)] = lv_apply_row(L, p, i, j, k);
}

static orc_level fine_level(const orc_grid *g, double *c)
{
    orc_level L;
    L.ndim = g->ndim;
    for (int a = 0; a < 3; ++a) { L.n[a] = g->n[a]; L.periodic[a] = a < g->ndim ? g->periodic[a] : 0; }
    L.c = c;
    return L;
}

void orc_poisson_apply(const orc_grid *g, const double *c, const double *p, double *Ap)
{
    orc_level L = fine_level(g, (double *)c);
    lv_apply(&L, p, Ap);
}

void orc_poisson_diag(const orc_grid *g, const double *c, double *D)
{
    orc_level L = fine_level(g, (double *)c);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < L.n[2]; ++k)
        for (int j = 0; j < L.n[1]; ++j)
            for (int i = 0; i < L.n[0]; ++i) D[lv_lin(&L, i, j, k)] = lv_diag(&L, i, j, k);
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid (Sec. 2, Sec. 4.2: MG with a PCG smoother).           */
/* Readings: halve every axis while all are even and all halves are >= 4;    */
/* restriction sums the 2^n children; the coarse face coefficient is half    */
/* the sum of the 2^(n-1) fine faces on it; prolongation is injection; the   */
/* cycle is V(0,k): k Jacobi-preconditioned CG iterations after the coarse   */
/* correction on every level; the coarsest level is solved by Jacobi-PCG to  */
/* round-off.                                                                */
/* ------------------------------------------------------------------------ */
#define OR_MAXLEV 24

static int can_coarsen(const orc_level *L)
{
    for (int a = 0; a < L->ndim; ++a)
        if ((L->n[a] % 2) != 0 || L->n[a] / 2 < 4) return 0;
    return 1;
}

static void coarsen(const orc_level *F, orc_level *C)
{
    C->ndim = F->ndim;
    for (int a = 0; a < 3; ++a) { C->n[a] = a < F->ndim ? F->n[a] / 2 : 1; C->periodic[a] = F->periodic[a]; }
    size_t ncc = lv_nc(C), ncf = lv_nc(F);
    C->c = (double *)calloc((size_t)C->ndim * ncc, sizeof(double));
    int kz = F->ndim == 3 ? 2 : 1;
    for (int a = 0; a < C->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < C->n[2]; ++k)
            for (int j = 0; j < C->n[1]; ++j)
                for (int i = 0; i < C->n[0]; ++i) {
                    double s = 0.0;
                    for (int oz = 0; oz < kz; ++oz)
                        for (int oy = 0; oy < 2; ++oy)
                            for (int ox = 0; ox < 2; ++ox) {
                                int o[3] = {ox, oy, oz};
                                if (o[a] != 0) continue;  /* fine faces on the coarse lower a-face */
                                s += F->c[(size_t)a * ncf + lv_lin(F, 2 * i + ox, 2 * j + oy, 2 * k + oz)];
                            }
                    C->c[(size_t)a * ncc + lv_lin(C, i, j, k)] = 0.5 * s;
                }
}

static void restrict_sum(const orc_level *F, const orc_level *C, const double *rf, double *rc)
{
    int kz = F->ndim == 3 ? 2 : 1;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < C->n[2]; ++k)
        for (int j = 0; j < C->n[1]; ++j)
            for (int i = 0; i < C->n[0]; ++i) {
                double s = 0.0;
                for (int oz = 0; oz < kz; ++oz)
                    for (int oy = 0; oy < 2; ++oy)
                        for (int ox = 0; ox < 2; ++ox) s += rf[lv_lin(F, 2 * i + ox, 2 * j + oy, 2 * k + oz)];
                rc[lv_lin(C, i, j, k)] = s;
            }
}

static void prolong_inject(const orc_level *F, const orc_level *C, const double *ec, double *ef)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < F->n[2]; ++k)
        for (int j = 0; j < F->n[1]; ++j)
            for (int i = 0; i < F->n[0]; ++i)
                ef[lv_lin(F, i, j, k)] = ec[lv_lin(C, i / 2, j / 2, F->ndim == 3 ? k / 2 : 0)];
}

/* Sums over a level in a fixed order that does not depend on the number of
 * threads: consecutive blocks of OR_RBLOCK terms are summed left to right
 * (blocks in parallel), then the block sums left to right. Below one block
 * this is the plain left-to-right sum. */
#define OR_RBLOCK 4096

/* sum_q w[q] a[q] b[q], with a NULL w counting every term once and a NULL b
 * taking b[q] = 1; w is a 0/1 mask (active rows) */
static double fixed_sum(const double *a, const double *b, const char *w, size_t n)
{
    size_t nb = (n + OR_RBLOCK - 1) / OR_RBLOCK;
    if (nb <= 1) {
        double s = 0.0;
        for (size_t q = 0; q < n; ++q)
            if (!w || w[q]) s += b ? a[q] * b[q] : a[q];
        return s;
    }
    double *part = malloc(nb * sizeof(double));
#pragma omp parallel for schedule(static)
    for (size_t blk = 0; blk < nb; ++blk) {
        size_t q1 = (blk + 1) * OR_RBLOCK < n ? (blk + 1) * OR_RBLOCK : n;
        double s = 0.0;
        for (size_t q = blk * OR_RBLOCK; q < q1; ++q)
            if (!w || w[q]) s += b ? a[q] * b[q] : a[q];
        part[blk] = s;
    }
    double s = 0.0;
    for (size_t blk = 0; blk < nb; ++blk) s += part[blk];
    free(part);
    return s;
}

static double dot(const double *a, const double *b, size_t n) { return fixed_sum(a, b, NULL, n); }

/* Jacobi-preconditioned CG on A x = r from the given x, for `iters` iterations
 * or until the residual norm falls to rtol * |r|. Rows with zero diagonal are
 * held fixed (their residual is zero by construction). */
static void pcg(const orc_level *L, const double *r, double *x, int iters, double rtol)
{
    size_t n = lv_nc(L);
    double *s = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
    double *d = malloc(n * sizeof(double)), *q = malloc(n * sizeof(double));
    double *iD = malloc(n * sizeof(double));
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < L->n[2]; ++k)
        for (int j = 0; j < L->n[1]; ++j)
            for (int i = 0; i < L->n[0]; ++i) {
                double D = lv_diag(L, i, j, k);
                iD[lv_lin(L, i, j, k)] = D != 0.0 ? 1.0 / D : 0.0;
            }
    lv_apply(L, x, q);
#pragma omp parallel for schedule(static)
    for (size_t e = 0; e < n; ++e) { s[e] = iD[e] != 0.0 ? r[e] - q[e] : 0.0; z[e] = iD[e] * s[e]; d[e] = z[e]; }
    double rho = dot(s, z, n);
    double r0 = sqrt(dot(r, r, n));
    for (int it = 0; it < iters; ++it) {
        if (rho == 0.0) break;
        if (rtol > 0.0 && sqrt(dot(s, s, n)) <= rtol * r0) break;
        lv_apply(L, d, q);
        double dq = dot(d, q, n);
        if (dq == 0.0) break;
        double alpha = rho / dq;
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < n; ++e) { x[e] += alpha * d[e]; s[e] -= alpha * q[e]; z[e] = iD[e] * s[e]; }
        double rho2 = dot(s, z, n);
        double beta = rho2 / rho;
        rho = rho2;
#pragma omp parallel for schedule(static)
        for (size_t e = 0; e < n; ++e) d[e] = z[e] + beta * d[e];
    }
    free(s); free(z); free(d); free(q); free(iD);
}

static void vcycle(orc_level *lev, int l, int nlev, const double *r, double *e, int k_smooth)
{
    size_t n = lv_nc(&lev[l]);
    if (l == nlev - 1) {
        /* The coarsest system is singular (periodic / Neumann boxes): solve for
         * the mean-free part of r over active rows, return a mean-free e. */
        double *rm = malloc(n * sizeof(double));
        char *act = malloc(n);
        double sr = 0.0, na = 0.0;
        orc_level *L = &lev[l];
        for (int k = 0; k < L->n[2]; ++k)
            for (int j = 0; j < L->n[1]; ++j)
                for (int i = 0; i < L->n[0]; ++i) {
                    size_t q = lv_lin(L, i, j, k);
                    act[q] = lv_diag(L, i, j, k) != 0.0;
                    if (act[q]) { sr += r[q]; na += 1.0; }
                }
        for (size_t q = 0; q < n; ++q) rm[q] = act[q] ? r[q] - sr / na : 0.0;
        memset(e, 0, n * sizeof(double));
        pcg(L, rm, e, 2 * (int)n + 200, 1e-14);
        double se = 0.0;
        for (size_t q = 0; q < n; ++q) if (act[q]) se += e[q];
        for (size_t q = 0; q < n; ++q) if (act[q]) e[q] -= se / na;
        free(rm); free(act);
        return;
    }
    size_t nc2 = lv_nc(&lev[l + 1]);
    double *rc = malloc(nc2 * sizeof(double)), *ec = malloc(nc2 * sizeof(double));
    restrict_sum(&lev[l], &lev[l + 1], r, rc);
    vcycle(lev, l + 1, nlev, rc, ec, k_smooth);
    prolong_inject(&lev[l], &lev[l + 1], ec, e);
    pcg(&lev[l], r, e, k_smooth, 0.0);
    free(rc); free(ec);
}

int orc_mg_levels(const orc_grid *g)
{
    orc_level L = fine_level(g, NULL);
    int nl = 1;
    while (can_coarsen(&L) && nl < OR_MAXLEV) {
        for (int a = 0; a < L.ndim; ++a) L.n[a] /= 2;
        ++nl;
    }
    return nl;
}

/* Solve A p = b - mean(b) for the pressure (warm start from p).
 * Readings: mean of b removed over active rows (nonzero diagonal); converged
 * when |b - A p|_2 <= tol |b|_2 over active rows; the returned p has zero mean
 * over active rows and zero on inactive rows. Returns 0, or 1 if not converged. */
int orc_poisson_solve(const orc_grid *g, const double *c, const double *b_in, double *p,
                      const orc_solver *S, orc_stats *st)
{
    orc_level lev[OR_MAXLEV];
    int nlev = 1;
    lev[0] = fine_level(g, (double *)c);
    while (can_coarsen(&lev[nlev - 1]) && nlev < OR_MAXLEV) {
        coarsen(&lev[nlev - 1], &lev[nlev]);
        ++nlev;
    }
    size_t n = lv_nc(&lev[0]);
    double *D = malloc(n * sizeof(double)), *b = malloc(n * sizeof(double));
    double *r = malloc(n * sizeof(double)), *e = malloc(n * sizeof(double));
    orc_poisson_diag(g, c, D);
    char *act = malloc(n);
    double na = 0.0;
    for (size_t q = 0; q < n; ++q) { act[q] = D[q] != 0.0; na += act[q] ? 1.0 : 0.0; }
    double sb = fixed_sum(b_in, NULL, act, n);
    double mean = na > 0 ? sb / na : 0.0;
    for (size_t q = 0; q < n; ++q) b[q] = D[q] != 0.0 ? b_in[q] - mean : 0.0;
    double bn = sqrt(dot(b, b, n));
    int it = 0, rc = 0;
    double rel = 0.0;
    for (;;) {
        lv_apply(&lev[0], p, r);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) r[q] = D[q] != 0.0 ? b[q] - r[q] : 0.0;
        double rn = sqrt(dot(r, r, n));
        rel = bn > 0.0 ? rn / bn : 0.0;
        if (rel <= S->tol) break;
        if (it >= S->itmax) { rc = 1; break; }
        vcycle(lev, 0, nlev, r, e, S->smooth_iters);
#pragma omp parallel for schedule(static)
        for (size_t q = 0; q < n; ++q) p[q] += e[q];
        ++it;
    }
    double sp = fixed_sum(p, NULL, act, n);
    double pm = na > 0 ? sp / na : 0.0;
    for (size_t q = 0; q < n; ++q) p[q] = D[q] != 0.0 ? p[q] - pm : 0.0;
    if (st) { st->vcycles = it; st->rel_resid = rel; st->bnorm = bn; }
    for (int l = 1; l < nlev; ++l) free(lev[l].c);
    free(D); free(b); free(r); free(e); free(act);
    return rc;
}

/* Pressure-gradient update u_a[I] -= w dt c_a[I] (p[I] - p[I-e_a]) (Sec. 3 listing). */
void orc_grad_update(const orc_grid *g, const double *c, const double *p, double wdt, double *u)
{
    size_t nc = ncell(g);
    orc_level L = fine_level(g, (double *)c);
    for (int a = 0; a < g->ndim; ++a)
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k}, Im[3] = {i, j, k};
                    Im[a] -= 1;
                    size_t q = (size_t)a * nc + lin(g, i, j, k);
                    u[q] -= wdt * c[q] * (p[lin(g, i, j, k)] - lv_p(&L, p, Im));
                    (void)I;
                }
}

/* Projection with weight w: A P = div(u)/(w dt), u -= w dt c grad P.
 * P is the warm start on entry and the solution on exit. */
int orc_project(const orc_grid *g, const double *c, double *u, const double *ue, double *P,
                double w, double dt, const orc_solver *S, orc_stats *st)
{
    size_t nc = ncell(g);
    double *b = malloc(nc * sizeof(double));
    orc_divergence(g, u, ue, b);
    double s = 1.0 / (w * dt);
    for (size_t q = 0; q < nc; ++q) b[q] *= s;
    int rc = orc_poisson_solve(g, c, b, P, S, st);
    orc_grad_update(g, c, P, w * dt, u);
    free(b);
    return rc;
}

/* CFL time step (Sec. 2: the time step adapts to keep the CFL number stable).
 * Reading: dt = min(dt_max, cfl / (max_I sum_a [max(0,u_a[I+e_a]) - min(0,u_a[I])] + 5 nu)). */
double orc_cfl(const orc_grid *g, const double *u, const double *ue, double cfl, double dt_max)
{
    double m = 0.0;
#pragma omp parallel for collapse(2) schedule(static) reduction(max : m)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double s = 0.0;
                for (int a = 0; a < g->ndim; ++a) {
                    int da[3] = {0, 0, 0};
                    da[a] = 1;
                    s += fmax(0.0, su(g, u, ue, a, i + da[0], j + da[1], k + da[2])) - fmin(0.0, su(g, u, ue, a, i, j, k));
                }
                if (s > m) m = s;
            }
    double dt = cfl / (m + 5.0 * g->nu);
    return dt < dt_max ? dt : dt_max;
}

/* Pressure force on the body (Sec. 5 reports drag, Sec. 6.1 power coefficients).
 * Reading: F = -sum_I p_I n(x_I) K_eps(d(x_I)) over cell centres (h^n = 1). */
void orc_forces(const orc_grid *g, const orc_body *B, double t, const double *p, double *F)
{
    F[0] = F[1] = F[2] = 0.0;
    if (B->kind == 0) return;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double x[3] = {i + 0.5, j + 0.5, k + 0.5};
                double d, nrm[3], v[3];
                orc_body_eval(B, g->ndim, x, t, &d, nrm, v);
                double K = orc_kernel(d, g->eps);
                if (K == 0.0) continue;
                double pk = p[lin(g, i, j, k)] * K;
                for (int a = 0; a < g->ndim; ++a) F[a] -= pk * nrm[a];
            }
}

/* Viscous force on the body (Sec. 5 reports drag; the paper prints no force
 * formula). Reading: the viscous traction nu (grad u + grad u^T) . n of the
 * stress on the body surface, n = grad d pointing into the fluid (the same
 * orientation as the pressure part -p n), spread over the kernel band:
 *   F_a = nu sum_I K_eps(d(x_I)) sum_b S_ab(x_I) n_b(x_I),  S = grad u + grad u^T,
 * the velocity gradient at the cell centre x_I from the face samples:
 *   d_a u_a = u_a[I+e_a] - u_a[I],
 *   d_b u_a = (u_a[I+e_b] + u_a[I+e_a+e_b] - u_a[I-e_b] - u_a[I+e_a-e_b]) / 4  (b != a),
 * samples beyond the stored range by the boundary rule of su. */
static double centre_grad(const orc_grid *g, const double *u, const double *ue, int a, int b, int i, int j, int k)
{
    int A[3] = {0, 0, 0}, Bv[3] = {0, 0, 0};
    A[a] = 1;
    Bv[b] = 1;
    if (a == b) return su(g, u, ue, a, i + A[0], j + A[1], k + A[2]) - su(g, u, ue, a, i, j, k);
    double up = su(g, u, ue, a, i + Bv[0], j + Bv[1], k + Bv[2]) +
                su(g, u, ue, a, i + A[0] + Bv[0], j + A[1] + Bv[1], k + A[2] + Bv[2]);
    double dn = su(g, u, ue, a, i - Bv[0], j - Bv[1], k - Bv[2]) +
                su(g, u, ue, a, i + A[0] - Bv[0], j + A[1] - Bv[1], k + A[2] - Bv[2]);
    return 0.25 * (up - dn);
}

void orc_forces_viscous(const orc_grid *g, const orc_body *B, double t, const double *u, const double *ue, double *F)
{
    F[0] = F[1] = F[2] = 0.0;
    if (B->kind == 0) return;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double x[3] = {i + 0.5, j + 0.5, k + 0.5};
                double d, nrm[3], v[3];
                orc_body_eval(B, g->ndim, x, t, &d, nrm, v);
                double K = orc_kernel(d, g->eps);
                if (K == 0.0) continue;
                double G[3][3] = {{0.0}};   /* G[a][b] = d_b u_a */
                for (int a = 0; a < g->ndim; ++a)
                    for (int b = 0; b < g->ndim; ++b) G[a][b] = centre_grad(g, u, ue, a, b, i, j, k);
                for (int a = 0; a < g->ndim; ++a) {
                    double tr = 0.0;
                    for (int b = 0; b < g->ndim; ++b) tr += (G[a][b] + G[b][a]) * nrm[b];
                    F[a] += g->nu * K * tr;
                }
            }
}

/* Derivative of the force component `axis` with respect to each cell's
 * pressure: the force is linear in p, dF_axis/dp_I = -n_axis(x_I) K_eps(d(x_I)). */
void orc_force_dp(const orc_grid *g, const orc_body *B, double t, int axis, double *out)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double x[3] = {i + 0.5, j + 0.5, k + 0.5};
                double d, nrm[3], v[3];
                out[lin(g, i, j, k)] = 0.0;
                if (B->kind == 0) continue;
                orc_body_eval(B, g->ndim, x, t, &d, nrm, v);
                out[lin(g, i, j, k)] = -nrm[axis] * orc_kernel(d, g->eps);
            }
}

/* Viscous force of a sampled body (the reading of orc_forces_viscous) with the
 * distance dc and normal ncen (component b at b*nc) sampled at the cell
 * centres. */
void orc_forces_viscous_sampled(const orc_grid *g, const double *dc, const double *ncen, const double *u,
                                const double *ue, double *F)
{
    size_t nc = ncell(g);
    F[0] = F[1] = F[2] = 0.0;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                size_t L = lin(g, i, j, k);
                double K = orc_kernel(dc[L], g->eps);
                if (K == 0.0) continue;
                double G[3][3] = {{0.0}};   /* G[a][b] = d_b u_a */
                for (int a = 0; a < g->ndim; ++a)
                    for (int b = 0; b < g->ndim; ++b) G[a][b] = centre_grad(g, u, ue, a, b, i, j, k);
                for (int a = 0; a < g->ndim; ++a) {
                    double tr = 0.0;
                    for (int b = 0; b < g->ndim; ++b) tr += (G[a][b] + G[b][a]) * ncen[(size_t)b * nc + L];
                    F[a] += g->nu * K * tr;
                }
            }
}

/* dF_axis/dp_I of the sampled body's pressure force: -n_axis K(d) at each
 * cell centre. */
void orc_force_dp_sampled(const orc_grid *g, const double *dc, const double *ncen, int axis, double *out)
{
    size_t nc = ncell(g);
    for (size_t L = 0; L < nc; ++L) out[L] = -ncen[(size_t)axis * nc + L] * orc_kernel(dc[L], g->eps);
}

/* One Heun predictor-corrector step with projections (Sec. 2), with the body
 * given by its measured face fields (mu0, mu1n, V; all NULL without a body).
 * State: u (ndim x nc), ue (exit plane), P (pressure, warm start in/out).
 *   u0 = u
 *   predictor:  u = B(u0 + dt R(u0)); BC; exit; project(w = 1)      -> u*
 *   corrector:  u = (u* + B(u0 + dt R(u*)))/2; BC; exit; project(w = 1/2)
 * Returns the number of projections that did not converge. */
int orc_step_fields(const orc_grid *g, const double *mu0, const double *mu1n, const double *V, double dt,
                    double *u, double *ue, double *P, const orc_solver *S, orc_stats *st2)
{
    size_t nc = ncell(g);
    size_t nu = (size_t)g->ndim * nc;
    int np = g->n[1] * g->n[2];
    double *u0 = malloc(nu * sizeof(double)), *r = malloc(nu * sizeof(double));
    double *ue0 = malloc((size_t)np * sizeof(double)), *ues = malloc((size_t)np * sizeof(double));
    double *c = malloc(nu * sizeof(double));
    orc_coeffs(g, mu0, c);
    memcpy(u0, u, nu * sizeof(double));
    memcpy(ue0, ue, (size_t)np * sizeof(double));
    int bad = 0;
    /* predictor */
    orc_conv_diff(g, u0, ue0, r);
    orc_bdim(g, u0, r, dt, mu0, mu1n, V, NULL, u);
    orc_exit_bc(g, ue0, u0, ue0, dt, 0, NULL, u, ue);
    bad += orc_project(g, c, u, ue, P, 1.0, dt, S, st2 ? &st2[0] : NULL);
    /* corrector */
    memcpy(ues, ue, (size_t)np * sizeof(double));
    orc_conv_diff(g, u, ue, r);
    double *us = malloc(nu * sizeof(double));
    memcpy(us, u, nu * sizeof(double));
    orc_bdim(g, u0, r, dt, mu0, mu1n, V, us, u);
    orc_exit_bc(g, ue0, us, ues, dt, 1, ues, u, ue);
    bad += orc_project(g, c, u, ue, P, 0.5, dt, S, st2 ? &st2[1] : NULL);
    free(us); free(u0); free(r); free(ue0); free(ues); free(c);
    return bad;
}

/* The step with the body measured at t + dt (the end of the step), held for
 * both stages. */
int orc_step(const orc_grid *g, const orc_body *B, double t, double dt,
             double *u, double *ue, double *P, const orc_solver *S, orc_stats *st2)
{
    size_t nc = ncell(g);
    size_t nu = (size_t)g->ndim * nc;
    double *mu0 = NULL, *mu1n = NULL, *V = NULL;
    if (B && B->kind != 0) {
        mu0 = malloc(nu * sizeof(double));
        mu1n = malloc(9 * nc * sizeof(double));
        V = malloc(nu * sizeof(double));
        orc_measure(g, B, t + dt, mu0, mu1n, V);
    }
    int bad = orc_step_fields(g, mu0, mu1n, V, dt, u, ue, P, S, st2);
    free(mu0); free(mu1n); free(V);
    return bad;
}

/* Diagnostics: kinetic energy (mean over cells of |u|^2/2 with u interpolated
 * to cell centres), and mean squared vorticity over cell edges (ν<|ω|²> is the
 * enstrophy form of the dissipation). */
void orc_diagnostics(const orc_grid *g, const double *u, const double *ue, double *ke, double *ens)
{
    double s = 0.0, w = 0.0;
    size_t nc = ncell(g);
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                int I[3] = {i, j, k};
                for (int a = 0; a < g->ndim; ++a) {
                    int da[3] = {0, 0, 0};
                    da[a] = 1;
                    double uc = 0.5 * (su(g, u, ue, a, i, j, k) + su(g, u, ue, a, i + da[0], j + da[1], k + da[2]));
                    s += 0.5 * uc * uc;
                }
                /* vorticity component about axis e on the edge at the lower corner:
                 * w_e = d_a u_b - d_b u_a, (a, b, e) cyclic */
                for (int e = 0; e < 3; ++e) {
                    int a = (e + 1) % 3, b = (e + 2) % 3;
                    if (g->ndim == 2 && e != 2) continue;
                    int ma[3] = {i, j, k}, mb[3] = {i, j, k};
                    ma[a] -= 1; mb[b] -= 1;
                    double om = (su(g, u, ue, b, i, j, k) - su(g, u, ue, b, ma[0], ma[1], ma[2]))
                              - (su(g, u, ue, a, i, j, k) - su(g, u, ue, a, mb[0], mb[1], mb[2]));
                    w += om * om;
                    (void)I;
                }
            }
    *ke = s / (double)nc;
    *ens = w / (double)nc;
}

/* ======================================================================== */
/* Discrete adjoint of one step (vector-Jacobian product) w.r.t. the start  */
/* velocity u0 and exit plane ue0, at fixed dt and fixed body, with the      */
/* limiter branches frozen at the evaluation point (subgradient at ties).    */
/* ======================================================================== */

/* Where a velocity sample comes from: kind 0 stored face (index into u),
 * 1 exit plane (index into ue), 2 constant. Mirrors su(). */
static void su_loc(const orc_grid *g, int a, int i, int j, int k, int *kind, size_t *index)
{
    int idx[3] = {i, j, k};
    int upper = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int N = g->n[ax];
        if (ax >= g->ndim) { idx[ax] = 0; continue; }
        if (g->periodic[ax]) idx[ax] = ((idx[ax] % N) + N) % N;
        else if (ax == a) {
            if (idx[ax] < 0) idx[ax] = 0;
            if (idx[ax] >= N) { idx[ax] = N; upper = 1; }
        } else {
            if (idx[ax] < 0) idx[ax] = 0;
            if (idx[ax] > N - 1) idx[ax] = N - 1;
        }
    }
    if (upper) {
        if (a == 0 && g->exit_hi_x) { *kind = 1; *index = (size_t)idx[1] + (size_t)g->n[1] * idx[2]; }
        else { *kind = 2; *index = 0; }
        return;
    }
    *kind = 0;
    *index = (size_t)a * ncell(g) + lin(g, idx[0], idx[1], idx[2]);
}

static void scatter(int kind, size_t index, double v, double *ub, double *ueb)
{
    if (kind == 0) ub[index] += v;
    else if (kind == 1) ueb[index] += v;
}

/* Transpose of the sampled body's viscous force (orc_forces_viscous_sampled)
 * contracted with w: the force is linear in the velocity samples, so
 * (ub, ueb) += d(w . F_v)/d(u, ue), each centre difference of centre_grad
 * passing its weight nu K (w_a n_b + w_b n_a) to the samples it reads. */
void orc_forces_viscous_sampled_vjp(const orc_grid *g, const double *dc, const double *ncen, const double *w,
                                    double *ub, double *ueb)
{
    size_t nc = ncell(g);
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                size_t L = lin(g, i, j, k);
                double K = orc_kernel(dc[L], g->eps);
                if (K == 0.0) continue;
                for (int a = 0; a < g->ndim; ++a)
                    for (int b = 0; b < g->ndim; ++b) {
                        double M = g->nu * K * (w[a] * ncen[(size_t)b * nc + L] + w[b] * ncen[(size_t)a * nc + L]);
                        int A[3] = {0, 0, 0}, Bv[3] = {0, 0, 0}, kind;
                        size_t at;
                        A[a] = 1;
                        Bv[b] = 1;
                        if (a == b) {
                            su_loc(g, a, i + A[0], j + A[1], k + A[2], &kind, &at);
                            scatter(kind, at, M, ub, ueb);
                            su_loc(g, a, i, j, k, &kind, &at);
                            scatter(kind, at, -M, ub, ueb);
                        } else {
                            double q = 0.25 * M;
                            su_loc(g, a, i + Bv[0], j + Bv[1], k + Bv[2], &kind, &at);
                            scatter(kind, at, q, ub, ueb);
                            su_loc(g, a, i + A[0] + Bv[0], j + A[1] + Bv[1], k + A[2] + Bv[2], &kind, &at);
                            scatter(kind, at, q, ub, ueb);
                            su_loc(g, a, i - Bv[0], j - Bv[1], k - Bv[2], &kind, &at);
                            scatter(kind, at, -q, ub, ueb);
                            su_loc(g, a, i + A[0] - Bv[0], j + A[1] - Bv[1], k + A[2] - Bv[2], &kind, &at);
                            scatter(kind, at, -q, ub, ueb);
                        }
                    }
            }
}

/* median3 with the index (0, 1, 2) of the argument it returns */
static double median3_w(double a, double b, double c, int *w)
{
    double m1 = a <= b ? a : b; int w1 = a <= b ? 0 : 1;
    double M1 = a <= b ? b : a; int wM = a <= b ? 1 : 0;
    double m2 = M1 <= c ? M1 : c; int w2 = M1 <= c ? wM : 2;
    if (m1 >= m2) { *w = w1; return m1; }
    *w = w2;
    return m2;
}

/* Partial derivatives of the limited QUICK value w.r.t. (uu, c, d). */
static double quick_d(double uu, double c, double d, double *g)
{
    double phi = (5.0 * c + 2.0 * d - uu) / 6.0;
    int wi, wo;
    double inner = median3_w(10.0 * c - 9.0 * uu, c, d, &wi);
    double val = median3_w(phi, c, inner, &wo);
    g[0] = g[1] = g[2] = 0.0;
    if (wo == 0) { g[0] = -1.0 / 6.0; g[1] = 5.0 / 6.0; g[2] = 2.0 / 6.0; }
    else if (wo == 1) g[1] = 1.0;
    else {
        if (wi == 0) { g[0] = -9.0; g[1] = 10.0; }
        else if (wi == 1) g[1] = 1.0;
        else g[2] = 1.0;
    }
    return val;
}

/* mu * dF/d(inputs) of the face flux of u_a through the lower b-face of the
 * control volume of cell I, scattered to the adjoint arrays. */
static void face_flux_vjp(const orc_grid *g, const double *u, const double *ue, int a, int b, int i, int j, int k,
                          double mu, double *ub, double *ueb)
{
    int db[3] = {0, 0, 0}, da[3] = {0, 0, 0};
    db[b] = 1; da[a] = 1;
    int P[6][3] = {{i, j, k}, {i - da[0], j - da[1], k - da[2]},
                   {i - 2 * db[0], j - 2 * db[1], k - 2 * db[2]}, {i - db[0], j - db[1], k - db[2]},
                   {i, j, k}, {i + db[0], j + db[1], k + db[2]}};
    int comp[6] = {b, b, a, a, a, a};
    double v[6];
    int kind[6];
    size_t ix[6];
    for (int q = 0; q < 6; ++q) {
        v[q] = su(g, u, ue, comp[q], P[q][0], P[q][1], P[q][2]);
        su_loc(g, comp[q], P[q][0], P[q][1], P[q][2], &kind[q], &ix[q]);
    }
    double Uf = 0.5 * (v[0] + v[1]);
    double gq[3], phi;
    /* (uu, c, d) = (sm2, sm1, s0) if Uf > 0 else (sp1, s0, sm1) */
    int map[3];
    if (Uf > 0.0) { phi = quick_d(v[2], v[3], v[4], gq); map[0] = 2; map[1] = 3; map[2] = 4; }
    else { phi = quick_d(v[5], v[4], v[3], gq); map[0] = 5; map[1] = 4; map[2] = 3; }
    scatter(kind[0], ix[0], mu * 0.5 * phi, ub, ueb);
    scatter(kind[1], ix[1], mu * 0.5 * phi, ub, ueb);
    for (int q = 0; q < 3; ++q) scatter(kind[map[q]], ix[map[q]], mu * Uf * gq[q], ub, ueb);
    scatter(kind[4], ix[4], -mu * g->nu, ub, ueb);
    scatter(kind[3], ix[3], mu * g->nu, ub, ueb);
}

/* (ub, ueb) += J_R(u, ue)^T lam */
void orc_conv_diff_vjp(const orc_grid *g, const double *u, const double *ue, const double *lam, double *ub, double *ueb)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    if (!g->periodic[a] && I[a] == 0) continue;
                    double l = lam[(size_t)a * nc + lin(g, i, j, k)];
                    if (l == 0.0) continue;
                    for (int b = 0; b < g->ndim; ++b) {
                        int db[3] = {0, 0, 0};
                        db[b] = 1;
                        face_flux_vjp(g, u, ue, a, b, i, j, k, l, ub, ueb);
                        face_flux_vjp(g, u, ue, a, b, i + db[0], j + db[1], k + db[2], -l, ub, ueb);
                    }
                }
}

/* fb += B^T gbar (blend transposed; boundary faces carry constants). */
static void bdim_vjp(const orc_grid *g, const double *mu0, const double *mu1n, const double *gbar, double *fb)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    if (!g->periodic[a] && I[a] == 0) continue;
                    size_t L = (size_t)a * nc + lin(g, i, j, k);
                    double gv = gbar[L];
                    if (!mu0) { fb[L] += gv; continue; }
                    fb[L] += mu0[L] * gv;
                    for (int b = 0; b < g->ndim; ++b) {
                        double m = mu1n[(size_t)(a * 3 + b) * nc + lin(g, i, j, k)];
                        if (m == 0.0) continue;
                        int P[3] = {i, j, k}, M[3] = {i, j, k};
                        P[b] += 1; M[b] -= 1;
                        for (int ax = 0; ax < 3; ++ax) {
                            if (ax >= g->ndim) continue;
                            int N = g->n[ax];
                            if (g->periodic[ax]) { P[ax] = ((P[ax] % N) + N) % N; M[ax] = ((M[ax] % N) + N) % N; }
                            else {
                                if (P[ax] > N - 1) P[ax] = N - 1;
                                if (M[ax] < 0) M[ax] = 0;
                            }
                        }
                        fb[(size_t)a * nc + lin(g, P[0], P[1], P[2])] += 0.5 * m * gv;
                        fb[(size_t)a * nc + lin(g, M[0], M[1], M[2])] -= 0.5 * m * gv;
                    }
                }
}

/* Exit condition transposed: given ueb_out, accumulate into ue0b, ueGb, uGb (last
 * interior x faces) and uesb (corrector). */
static void exit_vjp(const orc_grid *g, double dt, int corrector, const double *ueb_out, double *ue0b, double *ueGb,
                     double *uGb, double *uesb)
{
    if (!g->exit_hi_x) return;
    int np = g->n[1] * g->n[2], n0 = g->n[0];
    double m = 0.0;
    for (int p = 0; p < np; ++p) m += ueb_out[p];
    m /= np;
    double Ubar = g->U[0], w = corrector ? 0.5 : 1.0;
    for (int p = 0; p < np; ++p) {
        int j = p % g->n[1], k = p / g->n[1];
        double e = ueb_out[p] - m;
        ue0b[p] += w * e;
        ueGb[p] += -w * dt * Ubar * e;
        uGb[lin(g, n0 - 1, j, k)] += w * dt * Ubar * e;
        if (corrector) uesb[p] += 0.5 * e;
    }
}

/* Projection transposed: (ub, ueb) = (lu, le) + D^T q/(w dt), with
 * q = solve(lP - w dt G^T lu) (the solve's mean removal is symmetric); lP,
 * the cotangent of the returned pressure, may be NULL.
 * With the projection's own pressure P (u_out = u - w dt c grad P) and cb not
 * NULL, also the cotangent of the coefficients, through both the gradient
 * update and the operator A(c) (d(A^+ b) = -A^+ dA P):
 *   cb_a[I] += (P[I] - P[I-e_a]) ((q[I] - q[I-e_a]) - w dt lu_a[I])
 * on faces whose coefficient is the body's mu0 (not a non-periodic boundary). */
static void project_vjp(const orc_grid *g, const double *c, const double *lu, const double *le, const double *lP,
                        double w, double dt, double *ub, double *ueb, const double *P, double *cb)
{
    size_t nc = ncell(g);
    int np = g->n[1] * g->n[2];
    orc_level L = fine_level(g, (double *)c);
    double *rhs = calloc(nc, sizeof(double)), *q = calloc(nc, sizeof(double));
    double wdt = w * dt;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                int I[3] = {i, j, k};
                double s = 0.0;
                for (int a = 0; a < g->ndim; ++a) {
                    int Ip[3] = {i, j, k};
                    Ip[a] += 1;
                    s += c[(size_t)a * nc + lin(g, i, j, k)] * lu[(size_t)a * nc + lin(g, i, j, k)];
                    double cp = lv_c(&L, a, Ip);
                    if (cp != 0.0) {
                        int J[3] = {Ip[0], Ip[1], Ip[2]};
                        if (J[a] == g->n[a]) J[a] = 0;
                        s -= cp * lu[(size_t)a * nc + lin(g, J[0], J[1], J[2])];
                    }
                    (void)I;
                }
                rhs[lin(g, i, j, k)] = -wdt * s + (lP ? lP[lin(g, i, j, k)] : 0.0);
            }
    orc_solver S = {1e-13, 200, 4};
    orc_poisson_solve(g, c, rhs, q, &S, NULL);
    for (size_t e = 0; e < (size_t)g->ndim * nc; ++e) ub[e] = lu[e];
    for (int p = 0; p < np; ++p) ueb[p] = le ? le[p] : 0.0;
    for (int a = 0; a < g->ndim; ++a)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    int I[3] = {i, j, k};
                    size_t F = (size_t)a * nc + lin(g, i, j, k);
                    double qm = 0.0;
                    if (I[a] > 0 || g->periodic[a]) {
                        int M[3] = {i, j, k};
                        M[a] -= 1;
                        if (M[a] < 0) M[a] += g->n[a];
                        qm = q[lin(g, M[0], M[1], M[2])];
                    }
                    ub[F] += (qm - q[lin(g, i, j, k)]) / wdt;
                    if (a == 0 && g->exit_hi_x && i == g->n[0] - 1) ueb[j + g->n[1] * k] += q[lin(g, i, j, k)] / wdt;
                    if (cb && P && (I[a] > 0 || g->periodic[a])) {
                        int M[3] = {i, j, k};
                        M[a] -= 1;
                        if (M[a] < 0) M[a] += g->n[a];
                        double dP = P[lin(g, i, j, k)] - P[lin(g, M[0], M[1], M[2])];
                        cb[F] += dP * ((q[lin(g, i, j, k)] - qm) - wdt * lu[F]);
                    }
                }
    free(rhs); free(q);
}

/* Neighbour along b (dir = +1 or -1) of face (i,j,k), wrapped on periodic
 * axes and clamped to the stored range otherwise (the blend's samples). */
static size_t blend_nb(const orc_grid *g, int i, int j, int k, int b, int dir)
{
    int P[3] = {i, j, k};
    P[b] += dir;
    for (int ax = 0; ax < g->ndim; ++ax) {
        int N = g->n[ax];
        if (g->periodic[ax]) P[ax] = ((P[ax] % N) + N) % N;
        else if (P[ax] < 0) P[ax] = 0;
        else if (P[ax] > N - 1) P[ax] = N - 1;
    }
    return lin(g, P[0], P[1], P[2]);
}

/* Cotangents of the blend's face fields, given the blend input f and the
 * (masked) cotangent gbar of its output u = V + mu0 (f - V) + mu1 n.grad(f - V):
 *   mu0b += gbar (f - V);  mu1nb[a,b] += gbar (f - V)(P_b) - (f - V)(M_b)) / 2;
 *   Vb += gbar (1 - mu0), and the gradient term's -/+ gbar mu1 n_b / 2 at P_b / M_b. */
static void bdim_field_vjp(const orc_grid *g, const double *f, const double *mu0, const double *mu1n, const double *V,
                           const double *gbar, double *mu0b, double *mu1nb, double *Vb)
{
    size_t nc = ncell(g);
    for (int a = 0; a < g->ndim; ++a)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    size_t L = (size_t)a * nc + lin(g, i, j, k);
                    double gv = gbar[L];
                    if (gv == 0.0) continue;
                    mu0b[L] += gv * (f[L] - V[L]);
                    Vb[L] += gv * (1.0 - mu0[L]);
                    for (int b = 0; b < g->ndim; ++b) {
                        size_t up = (size_t)a * nc + blend_nb(g, i, j, k, b, +1);
                        size_t dn = (size_t)a * nc + blend_nb(g, i, j, k, b, -1);
                        size_t m = (size_t)(a * 3 + b) * nc + lin(g, i, j, k);
                        mu1nb[m] += gv * 0.5 * ((f[up] - V[up]) - (f[dn] - V[dn]));
                        Vb[up] -= gv * 0.5 * mu1n[m];
                        Vb[dn] += gv * 0.5 * mu1n[m];
                    }
                }
}

/* Vector-Jacobian product of orc_step_fields: given (lu, le, lP) for the
 * step's output (u, ue, P), return (ub, ueb) for its input (u0, ue0); lP may
 * be NULL. When mu0b, mu1nb, Vb are not NULL, the cotangents of the face
 * fields (mu0 through the blends and the Poisson coefficients, mu1 n, V) are
 * added to them (layout of orc_measure). The state arrays are not changed;
 * P0 (warm start) is used for the forward recomputation (the converged step
 * does not depend on it). */
void orc_step_vjp_fields(const orc_grid *g, const double *mu0, const double *mu1n, const double *V, double dt,
                         const double *u0, const double *ue0, const double *P0, const double *lu, const double *le,
                         const double *lP, double *ub, double *ueb, double *mu0b, double *mu1nb, double *Vb)
{
    size_t nc = ncell(g);
    size_t nu = (size_t)g->ndim * nc;
    int np = g->n[1] * g->n[2];
    int fields = mu0 && mu0b && mu1nb && Vb;
    double *c = malloc(nu * sizeof(double));
    orc_coeffs(g, mu0, c);
    orc_solver S = {1e-13, 200, 4};
    /* forward: predictor (u*, ue*, P1) and corrector (P2), keeping the blend inputs */
    double *r = malloc(nu * sizeof(double)), *us = malloc(nu * sizeof(double));
    double *f1 = malloc(nu * sizeof(double)), *f2 = malloc(nu * sizeof(double));
    double *ues = malloc((size_t)np * sizeof(double)), *P1 = malloc(nc * sizeof(double));
    double *P2 = malloc(nc * sizeof(double)), *u2 = malloc(nu * sizeof(double));
    double *ue2 = malloc((size_t)np * sizeof(double));
    memcpy(P1, P0, nc * sizeof(double));
    orc_conv_diff(g, u0, ue0, r);
    for (size_t e = 0; e < nu; ++e) f1[e] = u0[e] + dt * r[e];
    orc_bdim(g, u0, r, dt, mu0, mu1n, V, NULL, us);
    memcpy(ues, ue0, (size_t)np * sizeof(double));
    orc_exit_bc(g, ue0, u0, ue0, dt, 0, NULL, us, ues);
    orc_project(g, c, us, ues, P1, 1.0, dt, &S, NULL);
    if (fields) {
        orc_conv_diff(g, us, ues, r);
        for (size_t e = 0; e < nu; ++e) f2[e] = u0[e] + dt * r[e];
        orc_bdim(g, u0, r, dt, mu0, mu1n, V, us, u2);
        memcpy(ue2, ues, (size_t)np * sizeof(double));
        orc_exit_bc(g, ue0, us, ues, dt, 1, ues, u2, ue2);
        memcpy(P2, P1, nc * sizeof(double));
        orc_project(g, c, u2, ue2, P2, 0.5, dt, &S, NULL);
    }
    /* reverse */
    double *u2b = calloc(nu, sizeof(double)), *ue2b = calloc((size_t)np + 1, sizeof(double));
    double *usb = calloc(nu, sizeof(double)), *uesb = calloc((size_t)np + 1, sizeof(double));
    double *fb = calloc(nu, sizeof(double)), *u1b = calloc(nu, sizeof(double)), *ue1b = calloc((size_t)np + 1, sizeof(double));
    double *tmp = calloc(nu, sizeof(double));
    for (size_t e = 0; e < nu; ++e) ub[e] = 0.0;
    for (int p = 0; p < np; ++p) ueb[p] = 0.0;
    /* corrector projection (w = 1/2) */
    project_vjp(g, c, lu, le, lP, 0.5, dt, u2b, ue2b, fields ? P2 : NULL, fields ? mu0b : NULL);
    /* corrector exit: ue2 from ue0, ue*, u* */
    exit_vjp(g, dt, 1, ue2b, ueb, uesb, usb, uesb);
    /* corrector blend: u2 = (u* + B(u0 + dt R(u*)))/2 on non-boundary faces */
    for (int a = 0; a < g->ndim; ++a)
        for (size_t e = 0; e < nc; ++e) {
            size_t F = (size_t)a * nc + e;
            int i = (int)(e % g->n[0]), j = (int)((e / g->n[0]) % g->n[1]), k = (int)(e / ((size_t)g->n[0] * g->n[1]));
            int I[3] = {i, j, k};
            double v = (!g->periodic[a] && I[a] == 0) ? 0.0 : 0.5 * u2b[F];
            tmp[F] = v;
            usb[F] += v;
        }
    if (fields) bdim_field_vjp(g, f2, mu0, mu1n, V, tmp, mu0b, mu1nb, Vb);
    bdim_vjp(g, mu0, mu1n, tmp, fb);
    for (size_t e = 0; e < nu; ++e) { ub[e] += fb[e]; fb[e] *= dt; }
    orc_conv_diff_vjp(g, us, ues, fb, usb, uesb);
    /* predictor projection (w = 1) */
    project_vjp(g, c, usb, uesb, NULL, 1.0, dt, u1b, ue1b, fields ? P1 : NULL, fields ? mu0b : NULL);
    /* predictor exit: ue1 from ue0 (twice) and u0 */
    exit_vjp(g, dt, 0, ue1b, ueb, ueb, ub, NULL);
    /* predictor blend: u1 = B(u0 + dt R(u0)) */
    for (size_t e = 0; e < nu; ++e) { fb[e] = 0.0; tmp[e] = 0.0; }
    for (int a = 0; a < g->ndim; ++a)
        for (size_t e = 0; e < nc; ++e) {
            size_t F = (size_t)a * nc + e;
            int i = (int)(e % g->n[0]), j = (int)((e / g->n[0]) % g->n[1]), k = (int)(e / ((size_t)g->n[0] * g->n[1]));
            int I[3] = {i, j, k};
            tmp[F] = (!g->periodic[a] && I[a] == 0) ? 0.0 : u1b[F];
        }
    if (fields) bdim_field_vjp(g, f1, mu0, mu1n, V, tmp, mu0b, mu1nb, Vb);
    bdim_vjp(g, mu0, mu1n, tmp, fb);
    for (size_t e = 0; e < nu; ++e) { ub[e] += fb[e]; fb[e] *= dt; }
    orc_conv_diff_vjp(g, u0, ue0, fb, ub, ueb);
    free(c); free(r); free(us); free(f1); free(f2); free(ues); free(P1); free(P2); free(u2); free(ue2);
    free(u2b); free(ue2b); free(usb); free(uesb); free(fb); free(u1b); free(ue1b); free(tmp);
}

/* The same with the body measured at t + dt (as orc_step does). */
void orc_step_vjp(const orc_grid *g, const orc_body *B, double t, double dt, const double *u0, const double *ue0,
                  const double *P0, const double *lu, const double *le, const double *lP, double *ub, double *ueb)
{
    size_t nc = ncell(g);
    size_t nu = (size_t)g->ndim * nc;
    double *mu0 = NULL, *mu1n = NULL, *V = NULL;
    if (B && B->kind != 0) {
        mu0 = malloc(nu * sizeof(double)); mu1n = malloc(9 * nc * sizeof(double)); V = malloc(nu * sizeof(double));
        orc_measure(g, B, t + dt, mu0, mu1n, V);
    }
    orc_step_vjp_fields(g, mu0, mu1n, V, dt, u0, ue0, P0, lu, le, lP, ub, ueb, NULL, NULL, NULL);
    free(mu0); free(mu1n); free(V);
}
