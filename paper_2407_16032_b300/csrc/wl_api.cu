// wl_api.cu -- the C ABI of include/wl.h: argument checks, status codes and
// error strings around the simulation objects (wl_sim.cuh), plus the
// stand-alone network check entry point.
#include "../../include/wl.h"
#include "wl_sim_base.h"
#include "wl_common.cuh"
#include "k_net.cuh"
#include "k_net_tc.cuh"

#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using wl::Err;
using wl::SimBase;

namespace {

int validate(const wl_config *c, const wl_body *bd, std::string &msg) {
    if (!c) { msg = "cfg is NULL"; return WL_ERR_ARG; }
    if (c->ndim != 2 && c->ndim != 3) { msg = "ndim must be 2 or 3"; return WL_ERR_ARG; }
    for (int a = 0; a < c->ndim; ++a)
        if (c->n[a] < 2 || c->n[a] > (1 << 20)) { msg = "n[a] must be in [2, 2^20]"; return WL_ERR_ARG; }
    long long nc = 1;
    for (int a = 0; a < c->ndim; ++a) nc *= c->n[a];
    if (nc >= (1LL << 31)) { msg = "grid too large (the kernels index cells with 32-bit integers)"; return WL_ERR_ARG; }
    if (c->precision != WL_F32 && c->precision != WL_F64) { msg = "precision must be WL_F32 or WL_F64"; return WL_ERR_ARG; }
    if (!(c->eps > 0)) { msg = "eps must be positive"; return WL_ERR_ARG; }
    if (!(c->nu >= 0)) { msg = "nu must be >= 0"; return WL_ERR_ARG; }
    if (c->exit_hi_x && c->periodic[0]) { msg = "exit_hi_x needs a non-periodic x axis"; return WL_ERR_ARG; }
    if (!(c->tol > 0) || c->itmax < 0 || c->smooth_iters < 1 || c->smooth_iters > 64) { msg = "bad solver settings"; return WL_ERR_ARG; }
    if (!(c->dt_init > 0) || !(c->dt_max > 0) || !(c->cfl > 0)) { msg = "bad time-step settings"; return WL_ERR_ARG; }
    if (bd) {
        if (bd->kind < 0 || bd->kind > 4) { msg = "unknown body kind"; return WL_ERR_ARG; }
        if (bd->kind == WL_BODY_CYLINDER && c->ndim != 3) { msg = "cylinder body is 3D only (use a sphere in 2D)"; return WL_ERR_ARG; }
        if (bd->kind == WL_BODY_CYLINDER && !(bd->radius > 0)) { msg = "cylinder radius must be positive"; return WL_ERR_ARG; }
        if (bd->kind == WL_BODY_ELLIPSE && c->ndim != 2) { msg = "ellipse body is 2D only"; return WL_ERR_ARG; }
        if (bd->kind == WL_BODY_SPHERE && !(bd->radius > 0)) { msg = "sphere radius must be positive"; return WL_ERR_ARG; }
        if (bd->kind == WL_BODY_ELLIPSE && !(bd->semi[0] > 0 && bd->semi[1] > 0)) { msg = "ellipse semi-axes must be positive"; return WL_ERR_ARG; }
        if (bd->heave_axis < 0 || bd->heave_axis >= c->ndim) { msg = "heave_axis out of range"; return WL_ERR_ARG; }
    }
    return WL_OK;
}

}  // namespace

struct wl_sim {
    SimBase *impl;
    std::string err;
};

template <typename F>
static int guard(wl_sim *s, F &&f) {
    if (!s || !s->impl) return WL_ERR_ARG;
    try {
        int rc = f();
        s->err = rc == WL_OK ? std::string() : s->impl->err;
        return rc;
    } catch (const Err &e) {
        s->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        s->err = "host allocation failed";
        return WL_ERR_ALLOC;
    }
}

extern "C" {

void wl_config_default(wl_config *c, int ndim, const int *n) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->ndim = ndim;
    for (int a = 0; a < 3; ++a) c->n[a] = (n && a < ndim) ? n[a] : 1;
    c->eps = 1.0;
    c->precision = WL_F32;
    c->cfl = 1.0;
    c->dt_max = 1.0;
    c->dt_init = 0.25;
    c->dt_min = 1e-6;
    c->tol = 1e-6;
    c->itmax = 32;
    c->smooth_iters = 4;
}

int wl_sim_create(const wl_config *cfg, const wl_body *body, wl_sim **out) {
    if (!out) return WL_ERR_ARG;
    *out = nullptr;
    std::string msg;
    int rc = validate(cfg, body, msg);
    if (rc != WL_OK) { std::fprintf(stderr, "wl_sim_create: %s\n", msg.c_str()); return rc; }
    wl_sim *s = new (std::nothrow) wl_sim();
    if (!s) return WL_ERR_ALLOC;
    try {
        if (cfg->precision == WL_F64) s->impl = cfg->ndim == 3 ? wl::new_sim_f64_3d() : wl::new_sim_f64_2d();
        else s->impl = cfg->ndim == 3 ? wl::new_sim_f32_3d() : wl::new_sim_f32_2d();
        s->impl->init(*cfg, body);
    } catch (const Err &e) {
        std::fprintf(stderr, "wl_sim_create: %s\n", e.msg.c_str());
        delete s->impl;
        delete s;
        return e.code;
    } catch (const std::bad_alloc &) {
        delete s->impl;
        delete s;
        return WL_ERR_ALLOC;
    }
    *out = s;
    return WL_OK;
}

int wl_sim_destroy(wl_sim *s) {
    if (!s) return WL_OK;
    delete s->impl;
    delete s;
    return WL_OK;
}

int wl_set_velocity(wl_sim *s, const void *u, const void *ue) {
    if (!u) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->set_velocity(u, ue); return (int)WL_OK; });
}
int wl_get_velocity(wl_sim *s, void *u, void *ue) {
    if (!u) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->get_velocity(u, ue); return (int)WL_OK; });
}
int wl_get_pressure(wl_sim *s, double *p) {
    if (!p) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->get_pressure(p); return (int)WL_OK; });
}
int wl_set_pressure(wl_sim *s, const double *p) {
    if (!p) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->set_pressure(p); return (int)WL_OK; });
}
int wl_set_time(wl_sim *s, double t, double dt_next) {
    if (!(dt_next > 0)) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->t = t; s->impl->dt_next = dt_next; return (int)WL_OK; });
}
int wl_get_time(wl_sim *s, double *t, double *dt_next) {
    return guard(s, [&] {
        if (t) *t = s->impl->t;
        if (dt_next) *dt_next = s->impl->dt_next;
        return (int)WL_OK;
    });
}
int wl_mom_step(wl_sim *s, double dt_fixed, wl_step_stats *st) {
    return guard(s, [&] { return s->impl->mom_step(dt_fixed, st); });
}
int wl_project(wl_sim *s, double w, double dt, wl_solve_stats *st) {
    return guard(s, [&] { return s->impl->project(w, dt, st); });
}
int wl_poisson_solve(wl_sim *s, const void *b, double *p, wl_solve_stats *st) {
    if (!b || !p) return WL_ERR_ARG;
    return guard(s, [&] { return s->impl->poisson_solve(b, p, st); });
}
int wl_conv_diff(wl_sim *s, const void *u, const void *ue, void *r) {
    if (!u || !r) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->conv_diff(u, ue, r); return (int)WL_OK; });
}
int wl_forces(wl_sim *s, double *F) {
    if (!F) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->forces(F); return (int)WL_OK; });
}
int wl_forces_viscous(wl_sim *s, double *F) {
    if (!F) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->forces_viscous(F); return (int)WL_OK; });
}
int wl_body_update(wl_sim *s, double t) {
    return guard(s, [&] { s->impl->body_update(t); return (int)WL_OK; });
}
int wl_get_body_fields(wl_sim *s, void *c, void *mu1n, void *V) {
    return guard(s, [&] { s->impl->get_body_fields(c, mu1n, V); return (int)WL_OK; });
}
int wl_diagnostics(wl_sim *s, double *ke, double *ens, double *maxdiv) {
    return guard(s, [&] { s->impl->diagnostics(ke, ens, maxdiv); return (int)WL_OK; });
}
int wl_info(wl_sim *s, int *levels, long long *launches) {
    return guard(s, [&] { s->impl->info(levels, launches); return (int)WL_OK; });
}
int wl_profile(wl_sim *s, int on) {
    return guard(s, [&] { s->impl->profile(on); return (int)WL_OK; });
}
int wl_profile_report(wl_sim *s, char *buf, size_t len, size_t *needed) {
    return guard(s, [&] {
        std::string r = s->impl->profile_report();
        if (needed) *needed = r.size() + 1;
        if (buf && len > 0) {
            size_t n = r.size() < len - 1 ? r.size() : len - 1;
            std::memcpy(buf, r.data(), n);
            buf[n] = 0;
        }
        return (int)WL_OK;
    });
}
int wl_guess_setup(wl_sim *s, int level, int capacity) {
    return guard(s, [&] { s->impl->guess_setup(level, capacity); return (int)WL_OK; });
}
int wl_guess_mode(wl_sim *s, int collect, int use) {
    return guard(s, [&] { s->impl->guess_mode(collect, use); return (int)WL_OK; });
}
int wl_guess_train(wl_sim *s, int iters, double lr, int batch, unsigned seed, double *loss_first, double *loss_last) {
    if (iters < 1 || batch < 1 || !(lr > 0)) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->guess_train(iters, lr, batch, seed, loss_first, loss_last); return (int)WL_OK; });
}
int wl_guess_weights(wl_sim *s, const float *in, float *out) {
    return guard(s, [&] { s->impl->guess_weights(in, out); return (int)WL_OK; });
}
int wl_guess_info(wl_sim *s, int *level, int *samples, double *gain) {
    return guard(s, [&] { s->impl->guess_info(level, samples, gain); return (int)WL_OK; });
}

// One forward and backward pass of the network on a given sample (test entry).
int wl_net_eval(int ndim, const int *n, const float *w, const float *x, const float *t, float *y, float *dw,
                double *loss) {
    if ((ndim != 2 && ndim != 3) || !n || !w || !x) return WL_ERR_ARG;
    NetGrid ng{n[0], n[1], ndim == 3 ? n[2] : 1, 0};
    // the network kernels index voxel x channel in int: V * NET_C < 2^31
    if (ng.nx < 1 || ng.ny < 1 || ng.nz < 1 || (long long)ng.nx * ng.ny * ng.nz > WL_NET_MAX_VOXELS) return WL_ERR_ARG;
    ng.V = ng.nx * ng.ny * ng.nz;
    const size_t V = ng.V;
    std::vector<void *> bufs;
    bool ok = true;
    auto dal = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) { ok = false; return nullptr; }
        bufs.push_back(p);
        return p;
    };
    float *W = (float *)dal(3 * NET_WL * 4), *fx = (float *)dal(V * 4), *ft = (float *)dal(V * 4);
    float *Y = (float *)dal(V * NET_C * 4), *Z1 = (float *)dal(V * NET_C * 4), *Z2 = (float *)dal(V * NET_C * 4);
    float *G = (float *)dal(3 * NET_WL * 4), *yo = (float *)dal(V * 4);
    __nv_bfloat16 *Wf = (__nv_bfloat16 *)dal(3 * NET_WL * 2), *Wb = (__nv_bfloat16 *)dal(3 * NET_WL * 2);
    __nv_bfloat16 *A0 = (__nv_bfloat16 *)dal(V * NET_C * 2), *A1 = (__nv_bfloat16 *)dal(V * NET_C * 2);
    __nv_bfloat16 *A2 = (__nv_bfloat16 *)dal(V * NET_C * 2), *dY = (__nv_bfloat16 *)dal(V * NET_C * 2);
    double *dl = (double *)dal(2 * sizeof(double));
    int *es = (int *)dal(sizeof(int));   // bit 2: a tensor-core wait timed out
    int rc = ok ? WL_OK : WL_ERR_ALLOC;
    if (rc == WL_OK) {
        cudaMemcpy(W, w, 3 * NET_WL * 4, cudaMemcpyDefault);
        cudaMemcpy(fx, x, V * 4, cudaMemcpyDefault);
        if (t) cudaMemcpy(ft, t, V * 4, cudaMemcpyDefault);
        cudaMemset(G, 0, 3 * NET_WL * 4);
        cudaMemset(dl, 0, 2 * sizeof(double));
        cudaMemset(es, 0, sizeof(int));
        const int eb = (int)((V + 255) / 256), vb = (int)((V * NET_C + 255) / 256);
        const int wb = (int)((V + 1023) / 1024);
        const dim3 dwg(wb < 1 ? 1 : (wb > 512 ? 512 : wb), NET_TAPS);
        k_net_weights<<<(3 * NET_WL + 255) / 256, 256>>>(W, Wf, Wb);
        k_net_input<<<eb, 256>>>(ng.V, fx, A0);
        conv_fwd_tc(0, ng, A0, Wf, Z1, A1, es);
        conv_fwd_tc(0, ng, A1, Wf + NET_WL, Z2, A2, es);
        conv_fwd_tc(0, ng, A2, Wf + 2 * NET_WL, Y, nullptr, es);
        k_channel0<<<eb, 256>>>(ng.V, Y, yo);
        if (t) {
            k_sumsq<<<eb, 256>>>(ng.V, ft, dl + 1);
            k_net_loss<<<eb, 256>>>(ng.V, Y, ft, dl + 1, dY, dl);
            k_conv_dw<<<dwg, 128>>>(ng, A2, dY, G + 2 * NET_WL);
            conv_fwd_tc(0, ng, dY, Wb + 2 * NET_WL, Y, nullptr, es);
            k_relu_bwd<<<vb, 256>>>(ng.V * NET_C, Y, Z2, A2);
            k_conv_dw<<<dwg, 128>>>(ng, A1, A2, G + NET_WL);
            conv_fwd_tc(0, ng, A2, Wb + NET_WL, Y, nullptr, es);
            k_relu_bwd<<<vb, 256>>>(ng.V * NET_C, Y, Z1, A1);
            k_conv_dw<<<dwg, 128>>>(ng, A0, A1, G);
        }
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = WL_ERR_CUDA;
        int hes = 0;
        if (rc == WL_OK && (cudaMemcpy(&hes, es, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || hes)) rc = WL_ERR_CUDA;
        if (rc == WL_OK) {
            if (y) cudaMemcpy(y, yo, V * 4, cudaMemcpyDefault);
            if (dw && t) cudaMemcpy(dw, G, 3 * NET_WL * 4, cudaMemcpyDefault);
            if (loss && t) cudaMemcpy(loss, dl, sizeof(double), cudaMemcpyDeviceToHost);
        }
    }
    for (void *p : bufs) cudaFree(p);
    return rc;
}

int wl_step_vjp(wl_sim *s, double t, double dt, const void *u0, const void *ue0, const double *P0, const void *lu,
                const void *le, const double *lP, double tol, void *ub, void *ueb, wl_solve_stats *stats) {
    if (!u0 || !lu || !ub || !(tol > 0)) return WL_ERR_ARG;
    return guard(s, [&] { return s->impl->step_vjp(t, dt, u0, ue0, P0, lu, le, lP, tol, ub, ueb, stats); });
}
int wl_window_forward(wl_sim *s, int nsteps, int ckpt_every, const double *dts, const double *w, double *J,
                      double *dts_out) {
    return guard(s, [&] { return s->impl->window_forward(nsteps, ckpt_every, dts, w, nullptr, 0, J, dts_out); });
}
int wl_window_forward_weighted(wl_sim *s, int nsteps, int ckpt_every, const double *dts, const double *w,
                               const double *step_w, int viscous, double *J, double *dts_out) {
    return guard(s, [&] { return s->impl->window_forward(nsteps, ckpt_every, dts, w, step_w, viscous, J, dts_out); });
}
int wl_window_backward(wl_sim *s, double gJ, const void *lu, const void *le, double tol, void *du0, void *due0,
                       double *dparams) {
    if (!(tol > 0)) return WL_ERR_ARG;
    return guard(s, [&] { return s->impl->window_backward(gJ, lu, le, tol, du0, due0, dparams); });
}
int wl_tguess_mode(wl_sim *s, int collect, int use) {
    return guard(s, [&] { s->impl->tguess_mode(collect, use); return (int)WL_OK; });
}
int wl_tguess_fit(wl_sim *s, double *w, double *ratio) {
    return guard(s, [&] { s->impl->tguess_fit(w, ratio); return (int)WL_OK; });
}
int wl_tguess_weights(wl_sim *s, const double *in, double *out) {
    return guard(s, [&] { s->impl->tguess_weights(in, out); return (int)WL_OK; });
}
int wl_state_size(wl_sim *s, size_t *bytes) {
    if (!bytes) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->state_size(bytes); return (int)WL_OK; });
}
int wl_get_state(wl_sim *s, void *buf, size_t bytes) {
    if (!buf) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->get_state(buf, bytes); return (int)WL_OK; });
}
int wl_set_state(wl_sim *s, const void *buf, size_t bytes) {
    if (!buf) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->set_state(buf, bytes); return (int)WL_OK; });
}
int wl_window_stats(wl_sim *s, int *counts, double *max_rel) {
    return guard(s, [&] { s->impl->window_stats(counts, max_rel); return (int)WL_OK; });
}
int wl_set_body(wl_sim *s, const wl_body *body) {
    return guard(s, [&] { s->impl->set_body(body); return (int)WL_OK; });
}
int wl_set_coarse_dense_max(wl_sim *s, int max_cells) {
    return guard(s, [&] { s->impl->set_coarse_dense_max(max_cells); return (int)WL_OK; });
}
int wl_set_body_fields(wl_sim *s, const void *d_face, const void *n_face, const void *V_face, const void *d_cell,
                       const void *n_cell) {
    if (!d_face || !n_face || !V_face || !d_cell || !n_cell) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->set_body_fields(d_face, n_face, V_face, d_cell, n_cell); return (int)WL_OK; });
}
int wl_set_body_velocity_tangent(wl_sim *s, const void *dV_face) {
    return guard(s, [&] { s->impl->set_body_velocity_tangent(dV_face); return (int)WL_OK; });
}
int wl_force_dp(wl_sim *s, int axis, double scale, double *g) {
    if (!g) return WL_ERR_ARG;
    return guard(s, [&] { s->impl->force_dp(axis, scale, g); return (int)WL_OK; });
}

const char *wl_last_error(const wl_sim *s) { return s ? s->err.c_str() : "null sim"; }
const char *wl_status_string(int st) {
    switch (st) {
    case WL_OK: return "ok";
    case WL_ERR_ARG: return "invalid argument";
    case WL_ERR_CUDA: return "CUDA error";
    case WL_ERR_ALLOC: return "allocation failed";
    case WL_ERR_NOT_CONVERGED: return "Poisson solve not converged";
    case WL_ERR_NONFINITE: return "non-finite values";
    case WL_ERR_UNSTABLE: return "time step below dt_min";
    case WL_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

}  // extern "C"
