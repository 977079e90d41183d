// wl_sim_base.h -- the simulation interface shared by the per-precision
// translation units (wl_sim_*.cu) and the C ABI (wl_api.cu).
#pragma once
#include "../../include/wl.h"

#include <cuda_runtime.h>
#include <string>

namespace wl {

const double PI = 3.14159265358979323846;

struct Err {
    int code;
    std::string msg;
};

#define WL_CK(call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            throw Err{WL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};     \
        }                                                                                   \
    } while (0)

#define WL_LAUNCH_CK()                                                                      \
    do {                                                                                    \
        cudaError_t e_ = cudaGetLastError();                                                \
        if (e_ != cudaSuccess) throw Err{WL_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)}; \
    } while (0)

struct SimBase {
    wl_config cfg{};
    wl_body body{};
    std::string err;
    virtual ~SimBase() {}
    virtual void init(const wl_config &c, const wl_body *bd) = 0;
    virtual void set_velocity(const void *u, const void *ue) = 0;
    virtual void get_velocity(void *u, void *ue) = 0;
    virtual void get_pressure(double *p) = 0;
    virtual void set_pressure(const double *p) = 0;
    virtual int mom_step(double dt_fixed, wl_step_stats *st) = 0;
    virtual int project(double w, double dt, wl_solve_stats *st) = 0;
    virtual int poisson_solve(const void *b, double *p, wl_solve_stats *st) = 0;
    virtual void conv_diff(const void *u, const void *ue, void *r) = 0;
    virtual void forces(double *F) = 0;
    virtual void forces_viscous(double *F) = 0;
    virtual void body_update(double t) = 0;
    virtual void get_body_fields(void *c, void *mu1n, void *V) = 0;
    virtual void diagnostics(double *ke, double *ens, double *maxdiv) = 0;
    virtual void info(int *levels, long long *launches) = 0;
    virtual void profile(int on) = 0;
    virtual void guess_setup(int level, int capacity) = 0;
    virtual void guess_mode(int collect, int use) = 0;
    virtual void guess_train(int iters, double lr, int batch, unsigned seed, double *l0, double *l1) = 0;
    virtual void guess_weights(const float *in, float *out) = 0;
    virtual void guess_info(int *level, int *samples, double *gain) = 0;
    virtual std::string profile_report() = 0;
    virtual int step_vjp(double t0, double dt, const void *u0, const void *ue0, const double *P0, const void *lu,
                         const void *le, const double *lP, double tol, void *ub, void *ueb, wl_solve_stats *st) = 0;
    virtual void force_dp(int axis, double scale, double *g) = 0;
    virtual int window_forward(int nsteps, int ckpt, const double *dts, const double *w, const double *step_w,
                               int viscous, double *J, double *dts_out) = 0;
    virtual int window_backward(double gJ, const void *lu, const void *le, double tol, void *du0, void *due0,
                                double *dparams) = 0;
    virtual void set_body(const wl_body *bd) = 0;
    virtual void set_coarse_dense_max(int max_cells) = 0;
    virtual void window_stats(int *out4, double *max_rel) = 0;
    virtual void state_size(size_t *bytes) = 0;
    virtual void get_state(void *buf, size_t bytes) = 0;
    virtual void set_state(const void *buf, size_t bytes) = 0;
    virtual void set_body_fields(const void *d, const void *n, const void *V, const void *dc, const void *ncen) = 0;
    virtual void set_body_velocity_tangent(const void *dV) = 0;
    virtual void tguess_mode(int collect, int use) = 0;
    virtual void tguess_fit(double *w, double *ratio) = 0;
    virtual void tguess_weights(const double *in, double *out) = 0;
    double t = 0.0, dt_next = 0.25;
};


// One factory per (element type, dimension); each lives in its own
// translation unit so that the four instantiations compile in parallel.
SimBase *new_sim_f32_2d();
SimBase *new_sim_f32_3d();
SimBase *new_sim_f64_2d();
SimBase *new_sim_f64_3d();

}  // namespace wl
