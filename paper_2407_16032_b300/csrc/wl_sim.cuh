// wl_sim.cuh -- host driver of the BDIM time step: one simulation owns every
// device array of the step; the step enqueues its kernels on the caller's
// stream and reads back one small block of scalars per multigrid V-cycle
// (convergence test) and per step (time step, status). The V-cycle
// (restrictions, coarsest solve, prolongation + PCG smoothing on every level,
// and the next refinement residual) is one CUDA graph.
//
// Included once by each of wl_sim_{f32,f64}_{2d,3d}.cu, which instantiate
// Sim<T, ND> for one element type and dimension.
#pragma once
#include "wl_sim_base.h"
#include "wl_common.cuh"
#include "k_flux.cuh"
#include "k_body.cuh"
#include "k_poisson.cuh"
#include "k_coarse_dense.cuh"
#include "k_mg_march.cuh"
#include "k_resid.cuh"
#include "k_march4.cuh"
#include "k_flux4.cuh"
#include "k_misc.cuh"
#include "k_net.cuh"
#include "k_net_tc.cuh"
#include "k_adjoint.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <map>
#include <random>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

namespace wl {

// Per-kernel timing with CUDA events on the sim's stream (profiling mode only:
// the V-cycle then runs as direct launches instead of its graph).
struct Prof {
    struct Rec { const char *name; int level; long long cells; cudaEvent_t a, b; };
    bool on = false;
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::pair<std::string, int>, std::pair<long long, std::pair<double, long long>>> acc;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e;
        WL_CK(cudaEventCreate(&e));
        return e;
    }
    void beg(cudaStream_t s, const char *name, int level, long long cells) {
        if (!on) return;
        Rec r{name, level, cells, get(), get()};
        WL_CK(cudaEventRecord(r.a, s));
        pending.push_back(r);
    }
    void end(cudaStream_t s) {
        if (!on || pending.empty()) return;
        WL_CK(cudaEventRecord(pending.back().b, s));
    }
    void flush() {
        for (auto &r : pending) {
            WL_CK(cudaEventSynchronize(r.b));
            float ms = 0.f;
            WL_CK(cudaEventElapsedTime(&ms, r.a, r.b));
            auto &v = acc[{std::string(r.name), r.level}];
            v.first += 1;
            v.second.first += ms;
            v.second.second = r.cells;
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        pending.clear();
    }
    ~Prof() {
        for (auto &r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// A named NVTX range for the current scope (the step's phases on a profiler's
// timeline; without a tool attached the calls cost a few nanoseconds).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

template <typename T, int ND>
struct Sim : SimBase {
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;
    int nsm = 148, maxb = 1184;
    GridD g{};
    int nlev = 1;
    GridD gl[WL_MAXLEV];
    std::vector<void *> allocs;
    // fields
    T *vel[4][3] = {};
    int cur = 0;
    T *ueA = nullptr, *ueB = nullptr, *ueC = nullptr;
    T *mu1n = nullptr;
    T *Vb[3] = {};
    // refinement pressure (ph + pl), the warm start of every solve
    T *b = nullptr, *bl = nullptr, *ph = nullptr, *pl = nullptr;
    LevelD<T> lv[WL_MAXLEV];
    T *lc[WL_MAXLEV][3] = {};
    unsigned char *tfl[WL_MAXLEV] = {};
    double *cw = nullptr;   // coarsest scratch
    double *cM = nullptr;   // dense solution operator of the coarsest level
    bool cdense = false;
    int dense_max = 256;    // largest coarsest level (cells) solved by cM
    double *cMw = nullptr;  // scratch of its device build (moving bodies)
    int *tlist = nullptr;   // level-0 tiles flagged non-uniform (band blend)
    unsigned *tcount = nullptr;
    int *wlist = nullptr;   // weakly coupled level-0 rows (k_weak_list)
    unsigned *wcount = nullptr;
    double *pout = nullptr; // reported pressure scratch
    DevScalars *S = nullptr, *hS = nullptr;
    double *part = nullptr;
    cudaGraphExec_t vexec = nullptr;
    long long vnodes = 0;
    long long launches = 0;
    bool has_body = false, moving = false;
    // body given by caller samples (WL_BODY_USER_FACE_FIELDS): its cell-centre
    // distance and normal (forces), and an optional body-velocity tangent
    bool user = false, fields_set = false, vtan = false;
    T *dcell = nullptr, *ncell[3] = {}, *dVt[3] = {};
    double body_t = -1.0;
    bool measure_partial = false;   // the last measure updated a box only
    int np = 1;
    // learned initial guess (network on multigrid level gq.lev)
    struct GuessState {
        int lev = -1, shift = 0, cap = 0, count = 0, next = 0, step = 0;
        bool collect = false, use = false, ready = false;
        double gain = 1.0;
        NetGrid ng{};
        float *dx = nullptr, *dt = nullptr;  // samples: inputs, targets (cap x V)
        double *dn = nullptr;                 // per-sample sums of squares (x, t)
        float *W = nullptr, *G = nullptr, *m = nullptr, *v = nullptr, *Y = nullptr, *Z1 = nullptr, *Z2 = nullptr;
        float *fx = nullptr, *tt = nullptr;   // network input and scaled target (one sample)
        __nv_bfloat16 *Wf = nullptr, *Wb = nullptr, *A0 = nullptr, *A1 = nullptr, *A2 = nullptr, *dY = nullptr;
        double *loss = nullptr;
        int *tcst = nullptr;                  // bit 2: a tensor-core wait timed out during training
        T *ph0 = nullptr, *pl0 = nullptr;
    } gq;
    // adjoint of one step: forward copies, cotangents, and a backup of the state
    struct AdjState {
        bool ready = false, pready = false;
        T *u0[3] = {}, *us[3] = {}, *lu[3] = {}, *x[3] = {}, *usb[3] = {}, *fb[3] = {}, *ub[3] = {}, *bku[3] = {};
        T *ue0 = nullptr, *ues = nullptr, *le = nullptr, *xe = nullptr, *uesb = nullptr, *ueb = nullptr, *bkue = nullptr;
        T *bkph = nullptr, *bkpl = nullptr;
        double *lP = nullptr;
        // parameter mode: blend inputs and pressures of both stages, gradient
        T *f1[3] = {}, *f2[3] = {}, *P1h = nullptr, *P1l = nullptr, *P2h = nullptr, *P2l = nullptr;
        double *dpar = nullptr;
        // warm starts of the adjoint solves over a window (per stage: the
        // previous reverse step's solution)
        T *qh[2] = {}, *ql[2] = {};
        bool qwarm = false, qvalid[2] = {false, false};
    } ad;
    // learned temporal guess: per projection stage (0 predictor, 1 corrector)
    // its last two converged pressures (hi, lo), the fitted weights and the
    // gathered normal equations
    struct TGuess {
        bool collect = false, use = false, ready = false;
        T *H[2][2][2] = {};       // [stage][age][hi / lo]
        int count[2] = {0, 0};
        double w[2][2] = {{0.0, 1.0}, {0.0, 1.0}};
        double *stats = nullptr;  // 2 x 6 doubles on the device
    } tg;
    // checkpointed time window (forward run kept for the reverse sweep)
    struct Snap { T *u[3]; T *ue; T *ph; T *pl; double t; };
    struct Window {
        bool active = false;
        // adjoint solves of the last backward sweep: count, not converged,
        // largest V-cycle count, largest final relative residual, its step
        int solves = 0, unconverged = 0, max_vc = 0, worst_step = -1;
        double max_rel = 0.0;
        int n = 0, k = 0;
        double w[3] = {0, 0, 0};
        std::vector<double> dts, t0s, ws;   // steps, start times, per-step weights
        bool visc = false;                  // J includes the viscous force
        T *gv[3] = {}, *gve = nullptr;      // d(w . F_v)/d(u, ue) (constant for a fixed body)
        std::vector<Snap> ck, seg;
        Snap fin{};
        double fin_dt_next = 0.0;
    } win;
    Prof prof;
    void P0(const char *name, int level, long long cells) { prof.beg(st, name, level, cells); }
    void P1() { prof.end(st); }

    void *dalloc(size_t bytes) {
        void *p = nullptr;
        bytes = (bytes + 255) & ~size_t(255);
        if (cfg.allocator.alloc) {
            p = cfg.allocator.alloc(cfg.allocator.ctx, bytes);
            if (!p) throw Err{WL_ERR_ALLOC, "allocator callback returned NULL"};
        } else {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess) throw Err{WL_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        }
        allocs.push_back(p);
        WL_CK(cudaMemsetAsync(p, 0, bytes, st));
        return p;
    }
    template <typename Q> Q *alloc_n(size_t n) { return (Q *)dalloc(n * sizeof(Q)); }

    int blocks(long long n) const {
        long long b = (n + 255) / 256;
        return (int)(b < maxb ? (b < 1 ? 1 : b) : maxb);
    }
    // tiled kernels: one 32x8 block per tile, grid-stride over tiles
    int tgrid(int l) const { return lv[l].tl.nt < maxb ? lv[l].tl.nt : maxb; }
    dim3 tblk() const { return dim3(32, 8, 1); }

    ~Sim() override {
        if (vexec) cudaGraphExecDestroy(vexec);
        if (cap) cudaStreamDestroy(cap);
        if (hS) cudaFreeHost(hS);
        for (void *p : allocs) {
            if (cfg.allocator.alloc) {
                if (cfg.allocator.free) cfg.allocator.free(cfg.allocator.ctx, p);
            } else {
                cudaFree(p);
            }
        }
    }

    void init(const wl_config &c, const wl_body *bd) {
        cfg = c;
        st = (cudaStream_t)c.stream;
        if (bd) body = *bd; else { std::memset(&body, 0, sizeof(body)); body.kind = WL_BODY_NONE; }
        int dev = 0;
        WL_CK(cudaGetDevice(&dev));
        WL_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        maxb = nsm * 8;
        if (maxb > WL_MAXPART) maxb = WL_MAXPART;
        WL_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        WL_CK(cudaMallocHost(&hS, sizeof(DevScalars)));
        g.ndim = c.ndim;
        for (int a = 0; a < 3; ++a) {
            g.n[a] = (a < c.ndim) ? c.n[a] : 1;
            g.per[a] = (a < c.ndim) ? (c.periodic[a] != 0) : 0;
            g.U[a] = (a < c.ndim) ? c.U[a] : 0.0;
        }
        g.exit_x = c.exit_hi_x != 0;
        g.nu = c.nu;
        g.nc = (long long)g.n[0] * g.n[1] * g.n[2];
        np = g.n[1] * g.n[2];
        has_body = body.kind != WL_BODY_NONE;
        user = body.kind == WL_BODY_USER_FACE_FIELDS;
        moving = has_body && !user && (body.heave_amp != 0.0 || body.pitch_amp != 0.0);
        const long long nc = g.nc;
        for (int q = 0; q < 4; ++q)
            for (int a = 0; a < g.ndim; ++a) vel[q][a] = alloc_n<T>(nc);
        ueA = alloc_n<T>(np);
        ueB = alloc_n<T>(np);
        ueC = alloc_n<T>(np);
        if (has_body) {
            mu1n = alloc_n<T>((size_t)9 * nc);
            for (int a = 0; a < g.ndim; ++a) Vb[a] = alloc_n<T>(nc);
        }
        if (user) {
            dcell = alloc_n<T>(nc);
            for (int a = 0; a < g.ndim; ++a) ncell[a] = alloc_n<T>(nc);
        }
        b = alloc_n<T>(nc);
        bl = alloc_n<T>(nc);
        ph = alloc_n<T>(nc);
        pl = alloc_n<T>(nc);
        S = alloc_n<DevScalars>(1);
        part = alloc_n<double>(8 * WL_MAXPART);
        // multigrid hierarchy: halve every axis while all are even and >= 8
        gl[0] = g;
        nlev = 1;
        while (nlev < WL_MAXLEV) {
            const GridD &f = gl[nlev - 1];
            bool ok = true;
            for (int a = 0; a < g.ndim; ++a)
                if ((f.n[a] % 2) != 0 || f.n[a] / 2 < 4) ok = false;
            if (!ok) break;
            GridD cg = f;
            for (int a = 0; a < g.ndim; ++a) cg.n[a] = f.n[a] / 2;
            cg.nc = (long long)cg.n[0] * cg.n[1] * cg.n[2];
            gl[nlev++] = cg;
        }
        for (int l = 0; l < nlev; ++l) {
            const long long m = gl[l].nc;
            LevelD<T> &L = lv[l];
            L.g = gl[l];
            for (int a = 0; a < 3; ++a) {
                lc[l][a] = (a < g.ndim) ? alloc_n<T>(m) : nullptr;
                L.c[a] = lc[l][a];
            }
            L.invD = alloc_n<T>(m);
            L.x = alloc_n<T>(m);
            L.r = alloc_n<T>(m);
            L.s = alloc_n<T>(m);
            L.q = alloc_n<T>(m);
            L.d[0] = alloc_n<T>(m);
            L.d[1] = alloc_n<T>(m);
            L.tl = tiles_of(gl[l], MT<ND>::TZ);
            tfl[l] = alloc_n<unsigned char>(L.tl.nt);
            L.tflag = tfl[l];
            L.cu = (T)std::pow(2.0, (double)l * (ND - 2));
            // no body and every axis periodic: every cell has 2n faces of cu
            bool allper = true;
            for (int a = 0; a < g.ndim; ++a) allper = allper && g.per[a];
            L.iduni = (!has_body && allper) ? (T)(-1.0 / (2.0 * ND * (double)L.cu)) : T(0);
        }
        cw = alloc_n<double>(4 * gl[nlev - 1].nc);

        // initial state: u = 0 with U on boundary normal faces, exit plane U_x
        t = 0.0;
        dt_next = c.dt_init;
        set_velocity_fill();
        body_update(0.0);
        // a small coarsest level with coefficients that never change (no body
        // or a fixed one) is solved by a precomputed dense operator
        // the coarsest level (at most 256 cells) is solved by a dense solution
        // operator: built on the host once for fixed coefficients, on the
        // device after every measure of a moving body
        cdense = gl[nlev - 1].nc <= dense_max && coarse_dense();
        build_vcycle_graph();
        WL_CK(cudaStreamSynchronize(st));
    }

    // ------------------------------------------------------------ helpers
    CVec3P<T> cv(int q) const { CVec3P<T> r{}; for (int a = 0; a < 3; ++a) r.p[a] = vel[q][a]; return r; }
    Vec3P<T> vv(int q) const { Vec3P<T> r{}; for (int a = 0; a < 3; ++a) r.p[a] = vel[q][a]; return r; }
    CVec3P<T> cc0() const { CVec3P<T> r{}; for (int a = 0; a < 3; ++a) r.p[a] = lc[0][a]; return r; }

    void fill_boundary(int q) {
        k_bc_lower<T><<<blocks(g.nc), 256, 0, st>>>(g, vv(q));
        WL_LAUNCH_CK();
        ++launches;
    }

    void set_velocity_fill() {
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemsetAsync(vel[cur][a], 0, g.nc * sizeof(T), st));
        fill_boundary(cur);
        k_fill<T><<<blocks(np), 256, 0, st>>>((long long)np, (T)g.U[0], ueA);
        WL_LAUNCH_CK();
        ++launches;
    }

    BodyState body_state(double tt) const {
        BodyState B{};
        B.kind = body.kind;
        B.eps = cfg.eps;
        double c[3] = {body.centre[0], body.centre[1], body.centre[2]};
        double vc[3] = {0, 0, 0};
        const int ax = body.heave_axis;
        if (ax >= 0 && ax < 3) {
            c[ax] += body.heave_amp * std::sin(body.omega * tt + body.phase);
            vc[ax] = body.heave_amp * body.omega * std::cos(body.omega * tt + body.phase);
        }
        for (int a = 0; a < 3; ++a) {
            B.chi[a] = std::floor(c[a]);
            B.clo[a] = c[a] - B.chi[a];
            B.vc[a] = vc[a];
        }
        B.radius = body.radius;
        B.sa = body.semi[0];
        B.sb = body.semi[1];
        const double th = body.pitch_amp * std::sin(body.omega * tt + body.phase + 0.5 * PI);
        B.thd = body.pitch_amp * body.omega * std::cos(body.omega * tt + body.phase + 0.5 * PI);
        B.cth = std::cos(th);
        B.sth = std::sin(th);
        return B;
    }

    void read_scalars() {
        WL_CK(cudaMemcpyAsync(hS, S, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    // ------------------------------------------------------------ body
    // Box of level-0 cells whose measured fields can differ between the body
    // at time ta and at time tb: both positions' kernel bands and interiors
    // (the body's extent + eps + 3 cells around its centre; the band blend
    // reads the body velocity only there). False (measure everything) if the
    // box would wrap around a periodic axis.
    bool body_box(double ta, double tb, CellBox &b) const {
        double r;
        if (body.kind == WL_BODY_SPHERE || body.kind == WL_BODY_CYLINDER) r = body.radius;
        else if (body.kind == WL_BODY_ELLIPSE) r = std::max(body.semi[0], body.semi[1]);
        else return false;
        r += cfg.eps + 3.0;
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = 0;
            b.hi[a] = g.n[a];
            if (a >= ND || (body.kind == WL_BODY_CYLINDER && a == 2)) continue;
            double ca = body.centre[a], cb = body.centre[a];
            if (a == body.heave_axis) {
                ca += body.heave_amp * std::sin(body.omega * ta + body.phase);
                cb += body.heave_amp * std::sin(body.omega * tb + body.phase);
            }
            long long lo = (long long)std::floor(std::min(ca, cb) - r), hi = (long long)std::ceil(std::max(ca, cb) + r) + 1;
            if (lo < 0 || hi > g.n[a]) {
                if (g.per[a]) return false;
                lo = std::max(lo, 0LL);
                hi = std::min(hi, (long long)g.n[a]);
            }
            b.lo[a] = (int)lo;
            b.hi[a] = (int)hi;
        }
        return true;
    }
    // the level-0 box on level l, with a margin of one cell
    CellBox level_box(const CellBox &b0, int l) const {
        CellBox b{};
        for (int a = 0; a < 3; ++a) {
            if (a >= ND) { b.lo[a] = 0; b.hi[a] = 1; continue; }
            b.lo[a] = std::max(0, (b0.lo[a] >> l) - 1);
            b.hi[a] = std::min(gl[l].n[a], ((b0.hi[a] + (1 << l) - 1) >> l) + 1);
        }
        return b;
    }

    // A sampled body keeps its fields until the caller sets new ones: its
    // update only moves the time the fields stand for.
    void body_update(double tt) override {
        if (user && fields_set) { body_t = tt; return; }
        measure_body(tt, false);
    }

    // The coarsest level's dense solution operator for the current
    // coefficients: on the device where they change during a run (a moving or
    // sampled body) or where the level has more than 256 cells, else on the
    // host.
    bool coarse_dense() {
        return (moving || user || gl[nlev - 1].nc > 256) ? coarse_dense_device() : coarse_dense_build();
    }

    // A body given by samples (Sec. 3: distance function and map evaluated by
    // the caller): face distances d, face normals n (component b of face a at
    // slot a*ndim+b), face body velocities V, and the distance and normal at
    // the cell centres (forces). The moments, coefficients, 1/D and tile flags
    // of every level are formed on the device.
    void set_body_fields(const void *d, const void *n, const void *V, const void *dc, const void *ncen) override {
        if (!user) throw Err{WL_ERR_ARG, "set_body_fields: the body kind is not WL_BODY_USER_FACE_FIELDS"};
        if (!d || !n || !V || !dc || !ncen) throw Err{WL_ERR_ARG, "set_body_fields: a field pointer is NULL"};
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < ND; ++a) {
            WL_CK(cudaMemcpyAsync(lc[0][a], (const char *)d + a * bytes, bytes, cudaMemcpyDefault, st));
            WL_CK(cudaMemcpyAsync(Vb[a], (const char *)V + a * bytes, bytes, cudaMemcpyDefault, st));
            WL_CK(cudaMemcpyAsync(ncell[a], (const char *)ncen + a * bytes, bytes, cudaMemcpyDefault, st));
        }
        WL_CK(cudaMemcpyAsync(mu1n, n, (size_t)ND * ND * bytes, cudaMemcpyDefault, st));
        WL_CK(cudaMemcpyAsync(dcell, dc, bytes, cudaMemcpyDefault, st));
        Vec3P<T> c{};
        for (int a = 0; a < 3; ++a) c.p[a] = lc[0][a];
        P0("measure_sampled", 0, g.nc);
        k_measure_sampled<T, ND><<<blocks(g.nc), 256, 0, st>>>(g, c, mu1n, (long long)g.nc, cfg.eps);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        CellBox all{{0, 0, 0}, {g.n[0], g.n[1], g.n[2]}};
        levels_from_fine(all, false);
        body_t = t;
        measure_partial = false;
        fields_set = true;
        win.active = false;
        WL_CK(cudaStreamSynchronize(st));
    }

    // Tangent dV of the sampled body's face velocity along one parameter
    // (layout of V in set_body_fields); NULL clears it. The window gradient's
    // first parameter is then dJ/dtheta along it.
    void set_body_velocity_tangent(const void *dV) override {
        if (!user) throw Err{WL_ERR_ARG, "set_body_velocity_tangent: the body kind is not WL_BODY_USER_FACE_FIELDS"};
        vtan = dV != nullptr;
        if (!vtan) return;
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < ND; ++a) {
            if (!dVt[a]) dVt[a] = alloc_n<T>(g.nc);
            WL_CK(cudaMemcpyAsync(dVt[a], (const char *)dV + a * bytes, bytes, cudaMemcpyDefault, st));
        }
        WL_CK(cudaStreamSynchronize(st));
    }

    // Launch f with the cell-centre sampler of the body at time tt.
    template <typename F> void with_centre(double tt, F &&f) {
        if (user) {
            CentreSampled<T> cs{dcell, {ncell[0], ncell[1], ncell[2]}, cfg.eps};
            f(cs);
        } else {
            f(CentreAnalytic{body_state(tt)});
        }
    }

    // Measure the body at time tt onto the faces and rebuild the coefficients,
    // 1/D and tile flags of every level. partial: only inside the box where
    // the fields can differ from the last measure (at body_t, same body), the
    // per-step update of a moving body; the body velocity outside that box is
    // then left at its previous value (the step reads it only inside).
    void measure_body(double tt, bool partial) {
        Range rng("wl.measure");
        CellBox b0{};
        const bool box = partial && has_body && body_t >= 0 && body_box(body_t, tt, b0);
        if (!box)
            for (int a = 0; a < 3; ++a) { b0.lo[a] = 0; b0.hi[a] = a < ND ? g.n[a] : 1; }
        const long long bcells = (long long)(b0.hi[0] - b0.lo[0]) * (b0.hi[1] - b0.lo[1]) * (b0.hi[2] - b0.lo[2]);
        auto bgrid = [&](const CellBox &b, int l) {
            const long long nt = (long long)((b.hi[0] + 31) / 32 - b.lo[0] / 32) * ((b.hi[1] + 7) / 8 - b.lo[1] / 8) *
                                 ((b.hi[2] + MT<ND>::TZ - 1) / MT<ND>::TZ - b.lo[2] / MT<ND>::TZ);
            return (int)std::max(1LL, std::min(nt, (long long)maxb));
            (void)l;
        };
        BodyState B = body_state(tt);
        Vec3P<T> c{}, V{};
        for (int a = 0; a < 3; ++a) { c.p[a] = lc[0][a]; V.p[a] = Vb[a]; }
        P0("measure", 0, bcells);
        const int mgrid = (int)std::min<long long>((long long)bgrid(b0, 0) * MT<ND>::TZ, (long long)maxb);
        k_measure<T, ND><<<mgrid, tblk(), 0, st>>>(lv[0], B, c, mu1n, (long long)g.nc, V, has_body, b0);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        levels_from_fine(b0, box);
        body_t = tt;
        measure_partial = box;
    }

    // After the fine level's coefficients changed inside box b0 (everywhere
    // unless box): the coarse coefficients, 1/D and tile flags of every level,
    // the coarsest level's dense operator and the band blend's tile list.
    void levels_from_fine(const CellBox &b0, bool box) {
        auto bgrid = [&](const CellBox &b, int l) {
            const long long nt = (long long)((b.hi[0] + 31) / 32 - b.lo[0] / 32) * ((b.hi[1] + 7) / 8 - b.lo[1] / 8) *
                                 ((b.hi[2] + MT<ND>::TZ - 1) / MT<ND>::TZ - b.lo[2] / MT<ND>::TZ);
            return (int)std::max(1LL, std::min(nt, (long long)maxb));
            (void)l;
        };
        for (int l = 1; l < nlev; ++l) {
            CVec3P<T> cf{};
            Vec3P<T> cc{};
            for (int a = 0; a < 3; ++a) { cf.p[a] = lc[l - 1][a]; cc.p[a] = lc[l][a]; }
            const CellBox bl = box ? level_box(b0, l) : CellBox{{0, 0, 0}, {gl[l].n[0], gl[l].n[1], gl[l].n[2]}};
            k_coarsen_c<T, ND><<<bgrid(bl, l), tblk(), 0, st>>>(gl[l - 1], cf, lv[l], bl, cc);
            WL_LAUNCH_CK();
            ++launches;
        }
        for (int l = 0; l < nlev; ++l) {
            const CellBox bl = l == 0 ? b0 : (box ? level_box(b0, l) : CellBox{{0, 0, 0}, {gl[l].n[0], gl[l].n[1], gl[l].n[2]}});
            const long long cells = (long long)(bl.hi[0] - bl.lo[0]) * (bl.hi[1] - bl.lo[1]) * (bl.hi[2] - bl.lo[2]);
            if (l == 0) k_invd<T, ND, true><<<bgrid(bl, l), tblk(), 0, st>>>(lv[l], bl, (double)(g.nc - cells), S, part);
            else k_invd<T, ND, false><<<bgrid(bl, l), tblk(), 0, st>>>(lv[l], bl, 0.0, S, part);
            WL_LAUNCH_CK();
            k_tileflag_reset<ND><<<blocks(lv[l].tl.nt), 256, 0, st>>>(lv[l].tl, bl, tfl[l]);
            WL_LAUNCH_CK();
            k_tileflags<T, ND><<<bgrid(bl, l), tblk(), 0, st>>>(lv[l], bl, tfl[l]);
            WL_LAUNCH_CK();
            launches += 3;
        }
        if (cdense && (moving || user)) coarse_dense_device();
        // the level-0 tiles of the body (the band blend, the weak-row sweeps)
        if (has_body) {
            if (!tlist) {
                tlist = alloc_n<int>(lv[0].tl.nt);
                tcount = alloc_n<unsigned>(1);
            }
            WL_CK(cudaMemsetAsync(tcount, 0, sizeof(unsigned), st));
            k_tile_list<<<blocks(lv[0].tl.nt), 256, 0, st>>>(tfl[0], lv[0].tl.nt, tlist, tcount);
            WL_LAUNCH_CK();
            if (!wlist) {
                wlist = alloc_n<int>(g.nc);
                wcount = alloc_n<unsigned>(1);
            }
            WL_CK(cudaMemsetAsync(wcount, 0, sizeof(unsigned), st));
            k_weak_list<T, ND><<<nsm * 4, tblk(), 0, st>>>(lv[0], weak_cut(), tlist, tcount, wlist, wcount);
            WL_LAUNCH_CK();
            launches += 2;
        }
    }

    void get_body_fields(void *c, void *m1, void *V) override {
        if (measure_partial) measure_body(body_t, false);   // the body velocity everywhere
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < g.ndim; ++a) {
            if (c) WL_CK(cudaMemcpyAsync((char *)c + a * bytes, lc[0][a], bytes, cudaMemcpyDefault, st));
            if (V && has_body) WL_CK(cudaMemcpyAsync((char *)V + a * bytes, Vb[a], bytes, cudaMemcpyDefault, st));
        }
        if (m1 && has_body) WL_CK(cudaMemcpyAsync(m1, mu1n, 9 * bytes, cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    // ------------------------------------------------------------ multigrid
    void enqueue_vcycle(cudaStream_t s, long long &nodes) {
        const int k = cfg.smooth_iters;
        const bool tm = prof.on && s == st;
        auto B = [&](const char *nm, int l) { if (tm) P0(nm, l, gl[l].nc); };
        auto E = [&]() { if (tm) P1(); ++nodes; };
        // level 0 -> 1 restriction is fused into the refinement residual
        for (int l = 1; l + 1 < nlev; ++l) {
            B("restrict", l + 1);
            k_restrict<T, ND><<<tgrid(l + 1), tblk(), 0, s>>>(gl[l], lv[l].r, lv[l + 1]);
            E();
        }
        const int L = nlev - 1;
        long long ncl = gl[L].nc;
        int maxit = (int)(2 * ncl + 200);
        if (maxit > 2000) maxit = 2000;
        B("coarsest", L);
        if (cdense && ncl <= 256) k_coarsest_dense<T><<<1, 256, 0, s>>>(lv[L], cM);
        else if (cdense) {
            k_coarsest_dense_rows<T><<<(int)((ncl + 7) / 8), 256, 0, s>>>(lv[L], cM, cw);
            E();
            B("coarsest_fin", L);
            k_coarsest_dense_fin<T><<<1, 256, 0, s>>>(lv[L], cw);
        } else k_coarsest<T><<<1, ncl >= 512 ? 512 : 256, 0, s>>>(lv[L], cw, maxit);
        E();
        for (int l = nlev - 2; l >= 0; --l) {
            B("pcg_init", l);
            k_pcg_initm<T, ND><<<tgrid(l), tblk(), 0, s>>>(lv[l], gl[l + 1], lv[l + 1].x, S, part, l);
            E();
            for (int it = 0; it < k; ++it) {
                // d alternates between the two buffers (the next pass reads the
                // previous direction of neighbouring tiles while writing its own)
                T *dnew = lv[l].d[it & 1], *dold = lv[l].d[(it + 1) & 1];
                B(it == 0 ? "pcg_dq1" : "pcg_dq", l);
                dq_launch(l, it == 0, dold, dnew, s);
                E();
                const bool last = it == k - 1;
                B(last ? (l == 0 ? "pcg_u_last_fine" : "pcg_u_last") : "pcg_u", l);
                const int vb = blocks((gl[l].nc + 3) / 4);
                if (!last) k_pcg_u<T, false, false><<<vb, 256, 0, s>>>(lv[l], dnew, ph, pl, S, part, l, it);
                else if (l > 0) k_pcg_u<T, true, false><<<vb, 256, 0, s>>>(lv[l], dnew, ph, pl, S, part, l, it);
                else k_pcg_u<T, true, true><<<vb, 256, 0, s>>>(lv[l], dnew, ph, pl, S, part, l, it);
                E();
            }
        }
        if (nlev == 1) {
            B("padd", 0);
            k_padd<T><<<blocks(g.nc), 256, 0, s>>>(g, lv[0].x, ph, pl);
            E();
        }
        B("resid", 0);
        resid_launch(s);
        E();
    }

    // the fine level of FP32 3D grids whose rows split into 16-byte groups
    // marches planes (k_march4.cuh); coarser levels (too few tiles to fill
    // the GPU) and other grids run the column kernels
    bool march4(int l) const {
        return std::is_same<T, float>::value && ND == 3 && l == 0 && gl[l].n[0] % 4 == 0 && gl[l].n[0] >= 64;
    }
    int m4grid(int l, int per_sm = M4_MINB) const {
        const GridD &q = gl[l];
        const long long nt = (long long)((q.n[0] + m4::TX - 1) / m4::TX) * ((q.n[1] + m4::TY - 1) / m4::TY) *
                             ((q.n[2] + m4::KZ - 1) / m4::KZ);
        return (int)std::min<long long>(nt, (long long)nsm * per_sm);
    }
    void dq_launch(int l, bool first, const T *dold, T *dnew, cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value && ND == 3) {
            if (march4(l)) {
                static bool attr = false;
                if (!attr) {
                    WL_CK(cudaFuncSetAttribute(k_pcg_dq4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)pcg_dq4_smem<false>()));
                    attr = true;
                }
                if (first) k_pcg_dq4<true><<<m4grid(l), 256, pcg_dq4_smem<true>(), s>>>(lv[l], dold, dnew, S, part, l);
                else k_pcg_dq4<false><<<m4grid(l), 256, pcg_dq4_smem<false>(), s>>>(lv[l], dold, dnew, S, part, l);
                return;
            }
        }
        if (first) k_pcg_dq<T, ND, true><<<tgrid(l), tblk(), 0, s>>>(lv[l], dold, dnew, S, part, l);
        else k_pcg_dq<T, ND, false><<<tgrid(l), tblk(), 0, s>>>(lv[l], dold, dnew, S, part, l);
    }

    // refinement residual on level 0, restricted into level 1 when there is one
    void resid_launch(cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value && ND == 3) {
            if (march4(0)) {
                static bool attr = false;
                if (!attr) {
                    WL_CK(cudaFuncSetAttribute(k_resid4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)resid4_smem<true>()));
                    WL_CK(cudaFuncSetAttribute(k_resid4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)resid4_smem<false>()));
                    attr = true;
                }
                if (nlev > 1) k_resid4<true><<<m4grid(0, 2), 256, resid4_smem<true>(), s>>>(lv[0], b, bl, ph, pl, lv[1], S, part);
                else k_resid4<false><<<m4grid(0, 2), 256, resid4_smem<false>(), s>>>(lv[0], b, bl, ph, pl, lv[0], S, part);
                return;
            }
        }
        if (nlev > 1) k_residm<T, ND, true><<<tgrid(0), tblk(), 0, s>>>(lv[0], b, bl, ph, pl, lv[1], S, part);
        else k_residm<T, ND, false><<<tgrid(0), tblk(), 0, s>>>(lv[0], b, bl, ph, pl, lv[0], S, part);
    }

    // Dense solution operator of the coarsest level: the inverse of the active
    // operator bordered by the mean constraint, [A 1; 1^T 0], by Gauss-Jordan
    // elimination with partial pivoting in double on the host. Returns false
    // (PCG stays) if the bordered matrix is singular (a disconnected active set).
    bool coarse_dense_build() {
        const int L = nlev - 1;
        const GridD &cg = gl[L];
        const int n = (int)cg.nc;
        std::vector<T> hc[3], hinv(n);
        for (int a = 0; a < g.ndim; ++a) {
            hc[a].resize(n);
            WL_CK(cudaMemcpyAsync(hc[a].data(), lc[L][a], n * sizeof(T), cudaMemcpyDeviceToHost, st));
        }
        WL_CK(cudaMemcpyAsync(hinv.data(), lv[L].invD, n * sizeof(T), cudaMemcpyDeviceToHost, st));
        WL_CK(cudaStreamSynchronize(st));
        std::vector<int> act;
        std::vector<int> pos(n, -1);
        for (int e = 0; e < n; ++e)
            if (hinv[e] != T(0)) { pos[e] = (int)act.size(); act.push_back(e); }
        const int m = (int)act.size();
        if (m == 0) return false;
        const int K = m + 1;
        std::vector<double> A((size_t)K * K, 0.0), X((size_t)K * K, 0.0);
        const int st3[3] = {1, cg.n[0], cg.n[0] * cg.n[1]};
        double amax = 0.0;
        for (int r = 0; r < m; ++r) {
            const int e = act[r];
            const int I[3] = {e % cg.n[0], (e / cg.n[0]) % cg.n[1], e / (cg.n[0] * cg.n[1])};
            for (int a = 0; a < g.ndim; ++a) {
                const int N = cg.n[a];
                const bool per = cg.per[a] != 0;
                const int ep = I[a] == N - 1 ? (per ? e - (N - 1) * st3[a] : -1) : e + st3[a];
                const int em = I[a] == 0 ? (per ? e + (N - 1) * st3[a] : -1) : e - st3[a];
                const double cp = ep >= 0 ? (double)hc[a][ep] : 0.0, cm = (double)hc[a][e];
                A[(size_t)r * K + r] -= cp + cm;
                if (ep >= 0 && pos[ep] >= 0) A[(size_t)r * K + pos[ep]] += cp;
                if (em >= 0 && pos[em] >= 0) A[(size_t)r * K + pos[em]] += cm;
            }
            amax = std::max(amax, std::fabs(A[(size_t)r * K + r]));
            A[(size_t)r * K + m] = 1.0;
            A[(size_t)m * K + r] = 1.0;
        }
        for (int r = 0; r < K; ++r) X[(size_t)r * K + r] = 1.0;
        for (int c = 0; c < K; ++c) {
            int piv = c;
            for (int r = c + 1; r < K; ++r)
                if (std::fabs(A[(size_t)r * K + c]) > std::fabs(A[(size_t)piv * K + c])) piv = r;
            if (!(std::fabs(A[(size_t)piv * K + c]) > 1e-10 * std::max(amax, 1.0))) return false;
            if (piv != c)
                for (int q = 0; q < K; ++q) {
                    std::swap(A[(size_t)c * K + q], A[(size_t)piv * K + q]);
                    std::swap(X[(size_t)c * K + q], X[(size_t)piv * K + q]);
                }
            const double inv = 1.0 / A[(size_t)c * K + c];
            for (int q = 0; q < K; ++q) { A[(size_t)c * K + q] *= inv; X[(size_t)c * K + q] *= inv; }
            for (int r = 0; r < K; ++r) {
                if (r == c) continue;
                const double f = A[(size_t)r * K + c];
                if (f == 0.0) continue;
                for (int q = 0; q < K; ++q) {
                    A[(size_t)r * K + q] -= f * A[(size_t)c * K + q];
                    X[(size_t)r * K + q] -= f * X[(size_t)c * K + q];
                }
            }
        }
        std::vector<double> Mh((size_t)n * n, 0.0);
        for (int r = 0; r < m; ++r)
            for (int q = 0; q < m; ++q) Mh[(size_t)act[r] * n + act[q]] = X[(size_t)r * K + q];
        if (!cM) cM = alloc_n<double>((size_t)256 * 256);
        WL_CK(cudaMemcpyAsync(cM, Mh.data(), Mh.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        WL_CK(cudaStreamSynchronize(st));
        return true;
    }

    // Dense solution operator of the coarsest level from its current
    // coefficients, on the device (one PCG solve per column, all columns side
    // by side); enqueued on the sim's stream, so it follows the measure.
    bool coarse_dense_device() {
        const int L = nlev - 1;
        const long long n = gl[L].nc;
        if (n > dense_max || n > WL_DENSE_MAX) return false;
        const size_t nm = (size_t)std::max(n, 256LL);
        if (!cM) cM = alloc_n<double>(nm * nm);
        if (!cMw) cMw = alloc_n<double>((size_t)4 * n * n);
        int maxit = (int)(2 * n + 200);
        P0("coarse_operator", L, n);
        k_coarse_operator<T><<<(int)n, n >= 128 ? 128 : 64, 0, st>>>(lv[L], cM, cMw, maxit);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        return true;
    }

    void build_vcycle_graph() {
        if (vexec) {
            WL_CK(cudaGraphExecDestroy(vexec));
            vexec = nullptr;
        }
        cudaGraph_t graph;
        long long nodes = 0;
        WL_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        enqueue_vcycle(cap, nodes);
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (e != cudaSuccess) throw Err{WL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e)};
        WL_CK(cudaGraphInstantiate(&vexec, graph, 0));
        WL_CK(cudaGraphDestroy(graph));
        vnodes = nodes;
    }

    // b is in place; solve A (ph+pl) = b - mean with warm start; fills stats.
    int solve(wl_solve_stats *sts) {
        Range rng("wl.solve");
        P0("resid", 0, g.nc);
        resid_launch(st);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        const bool collecting = gq.collect && gq.cap > 0;
        if (collecting || (gq.use && gq.ready)) guess_begin(collecting);
        read_scalars();
        const double rel0 = hS->rel;
        int it = 0;
        while (hS->rel > cfg.tol && it < cfg.itmax && !(hS->status & 1)) {
            if (prof.on) {
                long long nodes = 0;
                enqueue_vcycle(st, nodes);
                WL_LAUNCH_CK();
                launches += nodes;
            } else {
                Range vr("wl.vcycle");
                WL_CK(cudaGraphLaunch(vexec, st));
                launches += vnodes;
            }
            read_scalars();
            ++it;
        }
        // status bit 2: the learned guess's tensor-core convolution gave up on a wait
        if (hS->status & 4) throw Err{WL_ERR_CUDA, "learned guess: a tensor-core convolution's wait timed out"};
        if (!(hS->status & 1)) weak_rows();
        if (sts) { sts->vcycles = it; sts->rel_resid = hS->rel; sts->bnorm = hS->bnorm; sts->rel_initial = rel0; }
        if (collecting && !(hS->status & 1) && hS->rel <= cfg.tol) guess_end();
        if (hS->status & 1) return WL_ERR_NONFINITE;
        if (hS->rel > cfg.tol) return WL_ERR_NOT_CONVERGED;
        return WL_OK;
    }

    // Gauss-Seidel sweeps over the weakly coupled rows of level 0 (faces
    // summing to less than half a face) after a solve (k_weak_rows): three
    // red-black sweeps; only a body makes such rows.
    double weak_cut() const { return 0.5 * (double)lv[0].cu; }
    void weak_rows() {
        if (!has_body) return;
        P0("weak_rows", 0, g.nc);
        for (int sweep = 0; sweep < 3; ++sweep)
            for (int colour = 0; colour < 2; ++colour)
                k_weak_rows<T, ND><<<nsm, 256, 0, st>>>(lv[0], b, bl, ph, pl, S, colour, wlist, wcount);
        P1();
        WL_LAUNCH_CK();
        launches += 6;
    }

    // status flags are per solve: clear them before its right-hand side is formed
    void clear_status() { WL_CK(cudaMemsetAsync(&S->status, 0, sizeof(int), st)); }

    int project_buf(int q, const T *ue, double w, double dt, wl_solve_stats *sts, int stage = -1) {
        Range rng("wl.project");
        clear_status();
        P0("div", 0, g.nc);
        k_div<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cv(q), ue, (T)(1.0 / (w * dt)), b, bl, S, part);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        const bool tgs = stage >= 0 && tg.ready;
        if (tgs && tg.use && tg.count[stage] >= 2 && tg.count[1 - stage] >= 1) tguess_apply(stage);
        int rc = solve(sts);
        if (tgs && rc == WL_OK) tguess_push(stage);
        P0("grad", 0, g.nc);
        k_grad<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], ph, pl, (T)(w * dt), vv(q));
        P1();
        WL_LAUNCH_CK();
        ++launches;
        return rc;
    }

    // ---------------------------------------------- learned temporal guess
    void tguess_alloc() {
        if (tg.ready) return;
        for (int sg = 0; sg < 2; ++sg)
            for (int a = 0; a < 2; ++a)
                for (int h = 0; h < 2; ++h) tg.H[sg][a][h] = alloc_n<T>(g.nc);
        tg.stats = alloc_n<double>(12);
        tg.ready = true;
    }
    void tguess_apply(int sg) {
        const int o = 1 - sg;
        P0("tguess_apply", 0, g.nc);
        k_tguess_apply<T><<<blocks(g.nc), 256, 0, st>>>(g.nc, tg.H[sg][0][0], tg.H[sg][0][1], tg.H[sg][1][0],
                                                        tg.H[sg][1][1], tg.H[o][0][0], tg.H[o][0][1],
                                                        (T)tg.w[sg][0], (T)tg.w[sg][1], ph, pl);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        // the solve that follows forms the guess's residual first
    }
    // after a converged projection of stage sg: gather the fit's normal
    // equations (collecting) and push the solution into the stage's history
    void tguess_push(int sg) {
        const int o = 1 - sg;
        if (tg.collect && tg.count[sg] >= 2 && tg.count[o] >= 1) {
            k_tguess_stats<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], ph, pl, tg.H[sg][0][0], tg.H[sg][0][1],
                                                               tg.H[sg][1][0], tg.H[sg][1][1], tg.H[o][0][0],
                                                               tg.H[o][0][1], S, part, tg.stats + 6 * sg);
            WL_LAUNCH_CK();
            ++launches;
        }
        std::swap(tg.H[sg][0][0], tg.H[sg][1][0]);
        std::swap(tg.H[sg][0][1], tg.H[sg][1][1]);
        WL_CK(cudaMemcpyAsync(tg.H[sg][0][0], ph, g.nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
        WL_CK(cudaMemcpyAsync(tg.H[sg][0][1], pl, g.nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
        if (tg.count[sg] < 2) ++tg.count[sg];
    }
    void tguess_mode(int collect, int use) override {
        tguess_alloc();
        if (collect && !tg.collect) WL_CK(cudaMemsetAsync(tg.stats, 0, 12 * sizeof(double), st));
        tg.collect = collect != 0;
        tg.use = use != 0;
        WL_CK(cudaStreamSynchronize(st));
    }
    // least-squares weights per stage from the gathered normal equations;
    // ratio[sg]: predicted initial-residual norm of the fitted guess over the
    // plain warm start's on the collected projections
    void tguess_fit(double *w, double *ratio) override {
        tguess_alloc();
        double h[12];
        WL_CK(cudaMemcpyAsync(h, tg.stats, sizeof(h), cudaMemcpyDeviceToHost, st));
        WL_CK(cudaStreamSynchronize(st));
        for (int sg = 0; sg < 2; ++sg) {
            const double *m = h + 6 * sg;
            const double G11 = m[0], G12 = m[1], G22 = m[2], c1 = m[3], c2 = m[4], dd = m[5];
            const double ridge = 1e-12 * (G11 + G22);
            const double a = G11 + ridge, d = G22 + ridge, det = a * d - G12 * G12;
            double w1 = 0.0, w2 = 1.0;
            if (det > 0 && G11 > 0 && G22 > 0) {
                w1 = (d * c1 - G12 * c2) / det;
                w2 = (a * c2 - G12 * c1) / det;
            }
            tg.w[sg][0] = w1;
            tg.w[sg][1] = w2;
            auto loss = [&](double x1, double x2) {
                return dd - 2 * (x1 * c1 + x2 * c2) + x1 * x1 * G11 + 2 * x1 * x2 * G12 + x2 * x2 * G22;
            };
            const double lp = loss(0.0, 1.0), lf = loss(w1, w2);
            if (w) { w[2 * sg] = w1; w[2 * sg + 1] = w2; }
            if (ratio) ratio[sg] = lp > 0 ? std::sqrt(std::max(lf, 0.0) / lp) : 1.0;
        }
    }
    void tguess_weights(const double *in, double *out) override {
        tguess_alloc();
        for (int q = 0; q < 4; ++q) {
            if (in) tg.w[q / 2][q % 2] = in[q];
            if (out) out[q] = tg.w[q / 2][q % 2];
        }
    }
    void tguess_reset() { tg.count[0] = tg.count[1] = 0; }

    // ------------------------------------------------------------ stages
    template <int NDIM, int MODE>
    void flux_launch(const FluxArgs<T> &A) {
        if constexpr (std::is_same<T, float>::value && NDIM == 3) {
            if (g.n[0] % 4 == 0 && g.n[0] >= 64) {
                static bool attr4 = false;
                if (!attr4) {
                    WL_CK(cudaFuncSetAttribute(k_flux4<MODE, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)f4::SMEM));
                    WL_CK(cudaFuncSetAttribute(k_flux4<MODE, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)f4::SMEM));
                    attr4 = true;
                }
                // 16-plane marches when they give every block a few tiles, else 8
                const long long nxy = (long long)((g.n[0] + f4::TX - 1) / f4::TX) * ((g.n[1] + f4::TY - 1) / f4::TY);
                const bool deep = nxy * ((g.n[2] + 15) / 16) >= 4LL * nsm * 2;
                const long long nt = nxy * (deep ? (g.n[2] + 15) / 16 : (g.n[2] + 7) / 8);
                const int grid = (int)std::min<long long>(nt, (long long)nsm * 2);
                static const char *names4[7] = {"flux_raw", "flux_pred_f", "flux_pred", "flux_corr_f", "flux_corr",
                                                "flux_pred_m", "flux_corr_m"};
                P0(names4[MODE], 0, g.nc);
                if (deep) k_flux4<MODE, 16><<<grid, 256, f4::SMEM, st>>>(g, A);
                else k_flux4<MODE, 8><<<grid, 256, f4::SMEM, st>>>(g, A);
                P1();
                WL_LAUNCH_CK();
                ++launches;
                return;
            }
        }
        if (MODE == FM_PRED_M || MODE == FM_CORR_M) throw Err{WL_ERR_CUDA, "mixed flux modes need the plane-marching kernel"};
        using TL = FluxTile<NDIM>;
        const size_t smem = (size_t)NDIM * TL::SN * sizeof(T);
        static bool attr = false;
        if (!attr) {
            WL_CK(cudaFuncSetAttribute(k_flux<T, NDIM, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr = true;
        }
        const long long ntiles = (long long)((g.n[0] + TL::TX - 1) / TL::TX) * ((g.n[1] + TL::TY - 1) / TL::TY) *
                                 ((g.n[2] + TL::TZ - 1) / TL::TZ);
        int occ = 0;
        WL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_flux<T, NDIM, MODE>, TL::NT, smem));
        if (occ < 1) occ = 1;
        long long grid = (long long)nsm * occ;
        if (grid > ntiles) grid = ntiles;
        dim3 blk(TL::TX, TL::TY, TL::TZ);
        static const char *names[7] = {"flux_raw", "flux_pred_f", "flux_pred", "flux_corr_f", "flux_corr",
                                       "flux_pred_m", "flux_corr_m"};
        P0(names[MODE], 0, g.nc);
        k_flux<T, NDIM, MODE><<<(int)grid, blk, smem, st>>>(g, A);
        P1();
        WL_LAUNCH_CK();
        ++launches;
    }
    template <int MODE>
    void flux(const FluxArgs<T> &A) {
        flux_launch<ND, MODE>(A);
    }

    FluxArgs<T> fargs(int qu, const T *ue, int qu0, int qout, double dt) {
        FluxArgs<T> A{};
        for (int a = 0; a < 3; ++a) {
            A.u[a] = vel[qu][a];
            A.u0[a] = qu0 >= 0 ? vel[qu0][a] : nullptr;
            A.out[a] = vel[qout][a];
        }
        A.ue = ue;
        A.dt = (T)dt;
        A.tflag = tfl[0];
        A.tntx = lv[0].tl.ntx;
        A.tnty = lv[0].tl.nty;
        return A;
    }

    // the flux kernel writes the stage's final value in tiles without a body
    // face and the blend runs on the other tiles only (FP32 3D grids of the
    // plane-marching flux kernel)
    bool band_blend() const {
        return std::is_same<T, float>::value && ND == 3 && has_body && g.n[0] % 4 == 0 && g.n[0] >= 64;
    }
    void blend_band(bool corr, int qf, int qstar, int qout) {
        CVec3P<T> f = cv(qf), V{}, us{};
        for (int a = 0; a < 3; ++a) { V.p[a] = Vb[a]; us.p[a] = qstar >= 0 ? vel[qstar][a] : nullptr; }
        P0("blend_band", 0, g.nc);
        const int gb = nsm * 4;
        if (corr) k_blend_band<T, ND, true><<<gb, tblk(), 0, st>>>(lv[0], f, mu1n, (long long)g.nc, V, us, vv(qout), tlist, tcount);
        else k_blend_band<T, ND, false><<<gb, tblk(), 0, st>>>(lv[0], f, mu1n, (long long)g.nc, V, us, vv(qout), tlist, tcount);
        P1();
        WL_LAUNCH_CK();
        P0("band_copy", 0, g.nc);
        k_band_copy<T, ND><<<gb, tblk(), 0, st>>>(lv[0], cv(qout), vv(qf), tlist, tcount);
        P1();
        WL_LAUNCH_CK();
        launches += 2;
    }

    void exit_stage(bool corr, int quG, double dt) {
        if (!g.exit_x) return;
        // ueB: start-of-step plane; ueC: star plane (corrector); result into ueA
        if (!corr) {
            P0("exit", 0, np);
            k_exit<T, false><<<1, 1024, 0, st>>>(g, ueB, vel[quG][0], ueB, nullptr, (T)dt, ueA);
            P1();
        } else {
            WL_CK(cudaMemcpyAsync(ueC, ueA, np * sizeof(T), cudaMemcpyDeviceToDevice, st));
            P0("exit", 0, np);
            k_exit<T, true><<<1, 1024, 0, st>>>(g, ueB, vel[quG][0], ueC, ueC, (T)dt, ueA);
            P1();
        }
        WL_LAUNCH_CK();
        ++launches;
    }

    void blend(bool corr, int qf, int qstar, int qout) {
        CVec3P<T> f = cv(qf), V{}, us{};
        for (int a = 0; a < 3; ++a) { V.p[a] = Vb[a]; us.p[a] = qstar >= 0 ? vel[qstar][a] : nullptr; }
        P0("blend", 0, g.nc);
        if (corr) k_blend<T, ND, true><<<tgrid(0), tblk(), 0, st>>>(lv[0], f, mu1n, (long long)g.nc, V, us, vv(qout));
        else k_blend<T, ND, false><<<tgrid(0), tblk(), 0, st>>>(lv[0], f, mu1n, (long long)g.nc, V, us, vv(qout));
        P1();
        WL_LAUNCH_CK();
        ++launches;
    }

    int mom_step(double dt_fixed, wl_step_stats *sts) override {
        Range rng("wl.step");
        const double dt = dt_fixed > 0 ? dt_fixed : dt_next;
        if (!(dt > cfg.dt_min)) throw Err{WL_ERR_UNSTABLE, "time step below dt_min"};
        if (moving) measure_body(t + dt, true);
        const int A0 = cur, B1 = (cur + 1) & 3, C2 = (cur + 2) & 3, D3 = (cur + 3) & 3;
        if (g.exit_x) WL_CK(cudaMemcpyAsync(ueB, ueA, np * sizeof(T), cudaMemcpyDeviceToDevice, st));
        wl_solve_stats s0{}, s1{};
        int rc0, rc1;
        int ustar, unew;
        const bool band = band_blend();
        nvtxRangePushA("wl.predictor");
        if (!has_body) {
            flux<FM_PRED_U>(fargs(A0, ueB, -1, B1, dt));
            ustar = B1;
        } else if (band) {
            flux<FM_PRED_M>(fargs(A0, ueB, -1, B1, dt));
            blend_band(false, B1, -1, C2);   // the body's tiles, blended through C2 back into B1
            ustar = B1;
        } else {
            flux<FM_PRED_F>(fargs(A0, ueB, -1, B1, dt));
            blend(false, B1, -1, C2);
            ustar = C2;
        }
        exit_stage(false, A0, dt);
        rc0 = project_buf(ustar, ueA, 1.0, dt, &s0, 0);
        nvtxRangePop();
        if (rc0 == WL_ERR_NONFINITE) return fail_restore(rc0, "non-finite values in the predictor projection");
        nvtxRangePushA("wl.corrector");
        if (!has_body) {
            flux<FM_CORR_U>(fargs(ustar, ueA, A0, C2, dt));
            unew = C2;
        } else if (band) {
            flux<FM_CORR_M>(fargs(ustar, ueA, A0, C2, dt));
            blend_band(true, C2, ustar, D3);   // through D3 back into C2
            unew = C2;
        } else {
            flux<FM_CORR_F>(fargs(ustar, ueA, A0, B1, dt));
            blend(true, B1, ustar, D3);
            unew = D3;
        }
        exit_stage(true, ustar, dt);
        rc1 = project_buf(unew, ueA, 0.5, dt, &s1, 1);
        nvtxRangePop();
        if (rc1 == WL_ERR_NONFINITE) return fail_restore(rc1, "non-finite values in the corrector projection");
        // CFL for the next step
        P0("cfl", 0, g.nc);
        k_cfl<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cv(unew), ueA, cfg.cfl, cfg.dt_max, S, part);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        read_scalars();
        prof.flush();
        cur = unew;
        t += dt;
        dt_next = hS->dt_next;
        if (sts) {
            sts->proj[0] = s0;
            sts->proj[1] = s1;
            sts->dt = dt;
            sts->t = t;
            sts->dt_next = dt_next;
        }
        if (!(dt_next == dt_next)) { err = "non-finite CFL time step"; return WL_ERR_NONFINITE; }
        if (rc0 != WL_OK || rc1 != WL_OK) { err = "Poisson solve did not reach tol within itmax"; return WL_ERR_NOT_CONVERGED; }
        if (dt_next < cfg.dt_min) { err = "CFL time step below dt_min"; return WL_ERR_UNSTABLE; }
        return WL_OK;
    }

    int fail_restore(int rc, const char *msg) {
        if (g.exit_x) WL_CK(cudaMemcpyAsync(ueA, ueB, np * sizeof(T), cudaMemcpyDeviceToDevice, st));
        WL_CK(cudaStreamSynchronize(st));
        err = msg;
        return rc;
    }

    int project(double w, double dt, wl_solve_stats *sts) override {
        if (!(w > 0 && dt > 0)) throw Err{WL_ERR_ARG, "project: w and dt must be positive"};
        int rc = project_buf(cur, ueA, w, dt, sts);
        WL_CK(cudaStreamSynchronize(st));
        return rc;
    }

    int poisson_solve(const void *bin, double *p, wl_solve_stats *sts) override {
        WL_CK(cudaMemcpyAsync(b, bin, g.nc * sizeof(T), cudaMemcpyDefault, st));
        WL_CK(cudaMemsetAsync(bl, 0, g.nc * sizeof(T), st));
        if (!pout) pout = alloc_n<double>(g.nc);
        WL_CK(cudaMemcpyAsync(pout, p, g.nc * sizeof(double), cudaMemcpyDefault, st));
        k_pin<T><<<blocks(g.nc), 256, 0, st>>>(g, pout, ph, pl);
        ++launches;
        clear_status();
        k_bstats<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], b, S, part);
        WL_LAUNCH_CK();
        ++launches;
        int rc = solve(sts);
        get_pressure(p);
        return rc;
    }

    void conv_diff(const void *u, const void *ue, void *r) override {
        const int qi = (cur + 1) & 3, qo = (cur + 2) & 3;
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemcpyAsync(vel[qi][a], (const char *)u + a * bytes, bytes, cudaMemcpyDefault, st));
        if (ue && g.exit_x) WL_CK(cudaMemcpyAsync(ueC, ue, np * sizeof(T), cudaMemcpyDefault, st));
        flux<FM_RAW>(fargs(qi, ueC, -1, qo, 1.0));
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemcpyAsync((char *)r + a * bytes, vel[qo][a], bytes, cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void set_velocity(const void *u, const void *ue) override {
        tguess_reset();
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemcpyAsync(vel[cur][a], (const char *)u + a * bytes, bytes, cudaMemcpyDefault, st));
        fill_boundary(cur);
        if (ue && g.exit_x) WL_CK(cudaMemcpyAsync(ueA, ue, np * sizeof(T), cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void get_velocity(void *u, void *ue) override {
        const size_t bytes = g.nc * sizeof(T);
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemcpyAsync((char *)u + a * bytes, vel[cur][a], bytes, cudaMemcpyDefault, st));
        if (ue && g.exit_x) WL_CK(cudaMemcpyAsync(ue, ueA, np * sizeof(T), cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void pmean() {
        k_pmean<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], ph, pl, S, part);
        WL_LAUNCH_CK();
        ++launches;
    }

    void get_pressure(double *p) override {
        if (!pout) pout = alloc_n<double>(g.nc);
        pmean();
        k_pout<T><<<blocks(g.nc), 256, 0, st>>>(g, ph, pl, lv[0].invD, S, pout);
        WL_LAUNCH_CK();
        ++launches;
        WL_CK(cudaMemcpyAsync(p, pout, g.nc * sizeof(double), cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void set_pressure(const double *p) override {
        tguess_reset();
        if (!pout) pout = alloc_n<double>(g.nc);
        WL_CK(cudaMemcpyAsync(pout, p, g.nc * sizeof(double), cudaMemcpyDefault, st));
        k_pin<T><<<blocks(g.nc), 256, 0, st>>>(g, pout, ph, pl);
        WL_LAUNCH_CK();
        ++launches;
        WL_CK(cudaStreamSynchronize(st));
    }

    void forces(double *F) override {
        F[0] = F[1] = F[2] = 0.0;
        if (!has_body) return;
        pmean();
        with_centre(body_t, [&](auto cs) {
            k_forces<T, decltype(cs)><<<blocks(g.nc), 256, 0, st>>>(g, cs, ph, pl, lv[0].invD, S, part);
        });
        WL_LAUNCH_CK();
        ++launches;
        read_scalars();
        F[0] = hS->red[0];
        F[1] = hS->red[1];
        F[2] = hS->red[2];
    }

    void forces_viscous(double *F) override {
        F[0] = F[1] = F[2] = 0.0;
        if (!has_body) return;
        with_centre(body_t, [&](auto cs) {
            k_forces_visc<T, decltype(cs)><<<blocks(g.nc), 256, 0, st>>>(g, cs, cv(cur), ueA, S, part);
        });
        WL_LAUNCH_CK();
        ++launches;
        read_scalars();
        F[0] = hS->red[0];
        F[1] = hS->red[1];
        F[2] = hS->red[2];
    }

    void diagnostics(double *ke, double *ens, double *maxdiv) override {
        k_diag<T><<<blocks(g.nc), 256, 0, st>>>(g, cv(cur), ueA, lv[0].invD, S, part);
        WL_LAUNCH_CK();
        ++launches;
        read_scalars();
        if (ke) *ke = hS->red[0];
        if (ens) *ens = hS->red[1];
        if (maxdiv) *maxdiv = hS->red[2];
    }

    void profile(int on) override {
        prof.flush();
        prof.on = on != 0;
        if (on) prof.acc.clear();
    }

    std::string profile_report() override {
        WL_CK(cudaStreamSynchronize(st));
        prof.flush();
        std::string out;
        char line[256];
        for (auto &kv : prof.acc) {
            std::snprintf(line, sizeof(line), "%s %d %lld %.6f %lld\n", kv.first.first.c_str(), kv.first.second,
                          kv.second.first, kv.second.second.first, kv.second.second.second);
            out += line;
        }
        return out;
    }

    // ---------------------------------------------------------- learned guess
    void guess_setup(int level, int capacity) override {
        if (level < 1 || level >= nlev) throw Err{WL_ERR_ARG, "guess level must be a coarse multigrid level"};
        if (capacity < 0 || capacity > 100000) throw Err{WL_ERR_ARG, "bad sample capacity"};
        if (gq.lev >= 0) throw Err{WL_ERR_STATE, "learned guess already set up"};
        if (gl[level].nc > WL_NET_MAX_VOXELS)
            throw Err{WL_ERR_ARG, "guess level too large for the network kernels (voxels x channels must stay below 2^31)"};
        gq.lev = level;
        gq.shift = level;
        gq.ng.nx = gl[level].n[0];
        gq.ng.ny = gl[level].n[1];
        gq.ng.nz = gl[level].n[2];
        gq.ng.V = (int)gl[level].nc;
        const size_t V = gq.ng.V;
        gq.cap = capacity;
        if (capacity > 0) {
            gq.dx = alloc_n<float>((size_t)capacity * V);
            gq.dt = alloc_n<float>((size_t)capacity * V);
            gq.dn = alloc_n<double>(2 * (size_t)capacity);
            gq.ph0 = alloc_n<T>(g.nc);
            gq.pl0 = alloc_n<T>(g.nc);
        }
        gq.W = alloc_n<float>(3 * NET_WL);
        gq.G = alloc_n<float>(3 * NET_WL);
        gq.m = alloc_n<float>(3 * NET_WL);
        gq.v = alloc_n<float>(3 * NET_WL);
        gq.Wf = alloc_n<__nv_bfloat16>(3 * NET_WL);
        gq.Wb = alloc_n<__nv_bfloat16>(3 * NET_WL);
        gq.fx = alloc_n<float>(V);
        gq.tt = alloc_n<float>(V);
        gq.Y = alloc_n<float>(V * NET_C);
        gq.Z1 = alloc_n<float>(V * NET_C);
        gq.Z2 = alloc_n<float>(V * NET_C);
        gq.A0 = alloc_n<__nv_bfloat16>(V * NET_C);
        gq.A1 = alloc_n<__nv_bfloat16>(V * NET_C);
        gq.A2 = alloc_n<__nv_bfloat16>(V * NET_C);
        gq.dY = alloc_n<__nv_bfloat16>(V * NET_C);
        gq.loss = alloc_n<double>(1);
        gq.tcst = alloc_n<int>(1);
        WL_CK(cudaStreamSynchronize(st));
    }

    void guess_mode(int collect, int use) override {
        if (gq.lev < 0) throw Err{WL_ERR_STATE, "learned guess not set up"};
        if (use && !gq.ready) throw Err{WL_ERR_STATE, "learned guess has no trained weights"};
        gq.collect = collect != 0;
        gq.use = use != 0;
    }

    void guess_weights(const float *in, float *out) override {
        if (gq.lev < 0) throw Err{WL_ERR_STATE, "learned guess not set up"};
        if (in) {
            WL_CK(cudaMemcpyAsync(gq.W, in, 3 * NET_WL * sizeof(float), cudaMemcpyDefault, st));
            k_net_weights<<<blocks(3 * NET_WL), 256, 0, st>>>(gq.W, gq.Wf, gq.Wb);
            WL_LAUNCH_CK();
            gq.ready = true;
        }
        if (out) WL_CK(cudaMemcpyAsync(out, gq.W, 3 * NET_WL * sizeof(float), cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void guess_info(int *level, int *samples, double *gain) override {
        if (level) *level = gq.lev;
        if (samples) *samples = gq.count;
        if (gain) *gain = gq.gain;
    }

    // restrict the current fine residual (already on level 1) down to the net level
    void restrict_to_guess_level() {
        for (int l = 1; l < gq.lev; ++l) {
            k_restrict<T, ND><<<tgrid(l + 1), tblk(), 0, st>>>(gl[l], lv[l].r, lv[l + 1]);
            WL_LAUNCH_CK();
            ++launches;
        }
    }

    // network forward on fx (FP32 input) -> Y (channel 0 = output)
    void net_forward(const float *x, int *status) {
        const NetGrid &ng = gq.ng;
        k_net_input<<<blocks(ng.V), 256, 0, st>>>(ng.V, x, gq.A0);
        conv_fwd_tc(st, ng, gq.A0, gq.Wf, gq.Z1, gq.A1, status);
        conv_fwd_tc(st, ng, gq.A1, gq.Wf + NET_WL, gq.Z2, gq.A2, status);
        conv_fwd_tc(st, ng, gq.A2, gq.Wf + 2 * NET_WL, gq.Y, nullptr, status);
        WL_LAUNCH_CK();
        launches += 4;
    }

    // At the start of a solve (after the first residual): record the sample
    // input and the warm start (collecting), or apply the network's correction
    // and recompute the residual (using).
    void guess_begin(bool collecting) {
        restrict_to_guess_level();
        const size_t V = gq.ng.V;
        if (collecting) {
            float *xs = gq.dx + (size_t)gq.next * V;
            if (sizeof(T) == sizeof(float)) WL_CK(cudaMemcpyAsync(xs, lv[gq.lev].r, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
            else k_to_float<T><<<blocks(V), 256, 0, st>>>((long long)V, lv[gq.lev].r, xs);
            WL_CK(cudaMemcpyAsync(gq.ph0, ph, g.nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
            WL_CK(cudaMemcpyAsync(gq.pl0, pl, g.nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
        } else {
            if (sizeof(T) == sizeof(float)) WL_CK(cudaMemcpyAsync(gq.fx, lv[gq.lev].r, V * sizeof(float), cudaMemcpyDeviceToDevice, st));
            else k_to_float<T><<<blocks(V), 256, 0, st>>>((long long)V, lv[gq.lev].r, gq.fx);
            P0("guess_net", gq.lev, (long long)V);
            net_forward(gq.fx, &S->status);
            P1();
            P0("guess_apply", 0, g.nc);
            k_guess_apply<T><<<blocks(g.nc), 256, 0, st>>>(g, gq.shift, gq.ng, (float)gq.gain, gq.Y, ph, pl);
            P1();
            P0("resid", 0, g.nc);
            resid_launch(st);
            P1();
            WL_LAUNCH_CK();
            launches += 3;
        }
    }

    // After a converged solve: the target (coarse mean of p_converged - p_warm),
    // mean-free, and the sample's norms.
    void guess_end() {
        const size_t V = gq.ng.V;
        float *ts = gq.dt + (size_t)gq.next * V;
        k_guess_target<T><<<blocks(V), 256, 0, st>>>(g, gq.shift, gq.ng, ph, pl, gq.ph0, gq.pl0, ts);
        k_demean<<<1, 1024, 0, st>>>(gq.ng.V, ts);
        WL_CK(cudaMemsetAsync(gq.dn + 2 * gq.next, 0, 2 * sizeof(double), st));
        k_sumsq<<<blocks(V), 256, 0, st>>>(gq.ng.V, gq.dx + (size_t)gq.next * V, gq.dn + 2 * gq.next);
        k_sumsq<<<blocks(V), 256, 0, st>>>(gq.ng.V, ts, gq.dn + 2 * gq.next + 1);
        WL_LAUNCH_CK();
        launches += 4;
        gq.next = (gq.next + 1) % gq.cap;
        if (gq.count < gq.cap) ++gq.count;
    }

    // Adam on the collected samples (inputs scaled to unit RMS, targets by the
    // same factor and by the dataset gain; the bias-free ReLU network is
    // positively homogeneous, so at inference y = gain * net(r)).
    void guess_train(int iters, double lr, int batch, unsigned seed, double *l0, double *l1) override {
        if (gq.lev < 0 || gq.count < 1) throw Err{WL_ERR_STATE, "no collected samples to train on"};
        const size_t V = gq.ng.V;
        const int n = gq.count;
        std::vector<double> hn(2 * n);
        WL_CK(cudaMemcpyAsync(hn.data(), gq.dn, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
        WL_CK(cudaStreamSynchronize(st));
        std::vector<double> ratio, sx(n);
        for (int i = 0; i < n; ++i) {
            sx[i] = std::sqrt(hn[2 * i] / V);
            if (hn[2 * i] > 0 && hn[2 * i + 1] > 0) ratio.push_back(std::sqrt(hn[2 * i + 1] / hn[2 * i]));
        }
        if (ratio.empty()) throw Err{WL_ERR_STATE, "collected samples are all zero"};
        std::nth_element(ratio.begin(), ratio.begin() + ratio.size() / 2, ratio.end());
        const double gain = ratio[ratio.size() / 2];
        std::vector<double> tn2(n);
        if (!gq.ready) {
            // He-style initial weights, seeded
            std::mt19937 rng(seed);
            std::normal_distribution<float> nd(0.f, 1.f);
            std::vector<float> w(3 * NET_WL, 0.f);
            for (int l = 0; l < 3; ++l)
                for (int t = 0; t < NET_TAPS; ++t)
                    for (int i = 0; i < NET_C; ++i)
                        for (int o = 0; o < NET_C; ++o) {
                            if ((l == 0 && i > 0) || (l == 2 && o > 0)) continue;
                            const float fan = (float)(NET_TAPS * (l == 0 ? 1 : NET_C));
                            w[(l * NET_TAPS + t) * NET_C * NET_C + i * NET_C + o] = nd(rng) * std::sqrt(2.f / fan);
                        }
            WL_CK(cudaMemcpyAsync(gq.W, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, st));
            WL_CK(cudaMemsetAsync(gq.m, 0, 3 * NET_WL * sizeof(float), st));
            WL_CK(cudaMemsetAsync(gq.v, 0, 3 * NET_WL * sizeof(float), st));
            gq.step = 0;
        }
        k_net_weights<<<blocks(3 * NET_WL), 256, 0, st>>>(gq.W, gq.Wf, gq.Wb);
        std::mt19937 pick(seed + 1);
        std::uniform_int_distribution<int> ud(0, n - 1);
        float *tt = gq.tt;
        double *dtn = gq.loss;
        std::vector<double> hl(1);
        double *tnorm = nullptr;
        tnorm = alloc_n<double>(1);
        const NetGrid &ng = gq.ng;
        const int wb = (ng.V + 16 * 4 * 16 - 1) / (16 * 4 * 16);
        WL_CK(cudaMemsetAsync(gq.tcst, 0, sizeof(int), st));
        const dim3 dwg(wb < 1 ? 1 : (wb > 512 ? 512 : wb), NET_TAPS);
        for (int itn = 0; itn < iters; ++itn) {
            WL_CK(cudaMemsetAsync(gq.G, 0, 3 * NET_WL * sizeof(float), st));
            WL_CK(cudaMemsetAsync(dtn, 0, sizeof(double), st));
            for (int bi = 0; bi < batch; ++bi) {
                const int sm = ud(pick);
                const float sxi = sx[sm] > 0 ? (float)(1.0 / sx[sm]) : 1.f;
                // input x / s, target t / (s gain)
                k_scale_copy<<<blocks(V), 256, 0, st>>>(ng.V, sxi, gq.dx + (size_t)sm * V, gq.fx);
                k_scale_copy<<<blocks(V), 256, 0, st>>>(ng.V, (float)(sxi / gain), gq.dt + (size_t)sm * V, tt);
                WL_CK(cudaMemsetAsync(tnorm, 0, sizeof(double), st));
                k_sumsq<<<blocks(V), 256, 0, st>>>(ng.V, tt, tnorm);
                net_forward(gq.fx, gq.tcst);
                k_net_loss<<<blocks(V), 256, 0, st>>>(ng.V, gq.Y, tt, tnorm, gq.dY, dtn);
                // layer 3
                k_conv_dw<<<dwg, 128, 0, st>>>(ng, gq.A2, gq.dY, gq.G + 2 * NET_WL);
                conv_fwd_tc(st, ng, gq.dY, gq.Wb + 2 * NET_WL, gq.Y, nullptr, gq.tcst);
                k_relu_bwd<<<blocks(V * NET_C), 256, 0, st>>>((int)(V * NET_C), gq.Y, gq.Z2, gq.A2);
                // layer 2 (A2 now holds dZ2)
                k_conv_dw<<<dwg, 128, 0, st>>>(ng, gq.A1, gq.A2, gq.G + NET_WL);
                conv_fwd_tc(st, ng, gq.A2, gq.Wb + NET_WL, gq.Y, nullptr, gq.tcst);
                k_relu_bwd<<<blocks(V * NET_C), 256, 0, st>>>((int)(V * NET_C), gq.Y, gq.Z1, gq.A1);
                // layer 1 (A1 now holds dZ1)
                k_conv_dw<<<dwg, 128, 0, st>>>(ng, gq.A0, gq.A1, gq.G);
                WL_LAUNCH_CK();
                launches += 14;
            }
            ++gq.step;
            k_adam<<<blocks(3 * NET_WL), 256, 0, st>>>(gq.W, gq.G, gq.m, gq.v, gq.step, (float)lr, (float)batch);
            k_net_weights<<<blocks(3 * NET_WL), 256, 0, st>>>(gq.W, gq.Wf, gq.Wb);
            WL_LAUNCH_CK();
            launches += 2;
            if (itn == 0 || itn == iters - 1) {
                WL_CK(cudaMemcpyAsync(hl.data(), dtn, sizeof(double), cudaMemcpyDeviceToHost, st));
                WL_CK(cudaStreamSynchronize(st));
                if (itn == 0 && l0) *l0 = hl[0] / batch;
                if (itn == iters - 1 && l1) *l1 = hl[0] / batch;
            }
        }
        int tcst = 0;
        WL_CK(cudaMemcpyAsync(&tcst, gq.tcst, sizeof(int), cudaMemcpyDeviceToHost, st));
        WL_CK(cudaStreamSynchronize(st));
        if (tcst) throw Err{WL_ERR_CUDA, "guess_train: a tensor-core convolution's wait timed out"};
        gq.gain = gain;
        gq.ready = true;
    }

    // ------------------------------------------------------------ adjoint
    void adj_alloc() {
        if (ad.ready) return;
        const long long nc = g.nc;
        for (int a = 0; a < g.ndim; ++a) {
            ad.u0[a] = alloc_n<T>(nc); ad.us[a] = alloc_n<T>(nc); ad.lu[a] = alloc_n<T>(nc);
            ad.x[a] = alloc_n<T>(nc); ad.usb[a] = alloc_n<T>(nc); ad.fb[a] = alloc_n<T>(nc);
            ad.ub[a] = alloc_n<T>(nc); ad.bku[a] = alloc_n<T>(nc);
        }
        ad.ue0 = alloc_n<T>(np); ad.ues = alloc_n<T>(np); ad.le = alloc_n<T>(np); ad.xe = alloc_n<T>(np);
        ad.uesb = alloc_n<T>(np); ad.ueb = alloc_n<T>(np); ad.bkue = alloc_n<T>(np);
        ad.bkph = alloc_n<T>(nc); ad.bkpl = alloc_n<T>(nc);
        ad.lP = alloc_n<double>(nc);
        ad.dpar = alloc_n<double>(2);
        for (int q = 0; q < 2; ++q) { ad.qh[q] = alloc_n<T>(nc); ad.ql[q] = alloc_n<T>(nc); }
        if (!pout) pout = alloc_n<double>(nc);
        ad.ready = true;
    }
    void adj_alloc_params() {
        adj_alloc();
        if (ad.pready) return;
        for (int a = 0; a < g.ndim; ++a) { ad.f1[a] = alloc_n<T>(g.nc); ad.f2[a] = alloc_n<T>(g.nc); }
        ad.P1h = alloc_n<T>(g.nc); ad.P1l = alloc_n<T>(g.nc); ad.P2h = alloc_n<T>(g.nc); ad.P2l = alloc_n<T>(g.nc);
        ad.pready = true;
    }
    static CVec3P<T> cvp(T *const (&p)[3]) { CVec3P<T> r{}; for (int a = 0; a < 3; ++a) r.p[a] = p[a]; return r; }
    static Vec3P<T> vvp(T *const (&p)[3]) { Vec3P<T> r{}; for (int a = 0; a < 3; ++a) r.p[a] = p[a]; return r; }
    void zero_vec(T *const (&p)[3]) {
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemsetAsync(p[a], 0, g.nc * sizeof(T), st));
    }
    void copy_vec(T *const (&dst)[3], T *const (&src)[3]) {
        for (int a = 0; a < g.ndim; ++a)
            WL_CK(cudaMemcpyAsync(dst[a], src[a], g.nc * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }
    void dcopy(T *dst, const T *src, size_t n) {
        WL_CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    }

    // Tangents of the body state at time tt along the heave and pitch amplitudes.
    void param_tangents(double tt, BodyTangent &h, BodyTangent &p) const {
        std::memset(&h, 0, sizeof(h));
        std::memset(&p, 0, sizeof(p));
        const int ax = body.heave_axis;
        if (ax >= 0 && ax < 3) {
            h.dc[ax] = std::sin(body.omega * tt + body.phase);
            h.dvc[ax] = body.omega * std::cos(body.omega * tt + body.phase);
        }
        if (body.kind == WL_BODY_ELLIPSE) {
            p.dth = std::sin(body.omega * tt + body.phase + 0.5 * PI);
            p.dthd = body.omega * std::cos(body.omega * tt + body.phase + 0.5 * PI);
        }
    }

    // Projection transposed: (out, oute) = (lam, le) + D^T A^+ (div(c lam) + lP/(w dt)).
    // With the stage's forward pressure (Ph, Pl) and params, also the
    // coefficient part of the parameter gradient.
    int proj_vjp(T *const (&lam)[3], const T *le, const double *lP, double w, double dt, T *const (&out)[3], T *oute,
                 wl_solve_stats *sts, const T *Ph = nullptr, const T *Pl = nullptr, const BodyTangent *dB = nullptr,
                 double tt = 0.0, int stage = -1) {
        P0("adj_rhs", 0, g.nc);
        k_adj_rhs<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cvp(lam), lP, 1.0 / (w * dt), b, bl);
        P1();
        clear_status();
        k_bstats<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], b, S, part);
        WL_LAUNCH_CK();
        launches += 2;
        // warm start: the same stage's solution of the previous reverse step
        // over a window (any start converges to the same solution), else 0
        const bool warm = stage >= 0 && ad.qwarm && ad.qvalid[stage];
        if (warm) {
            dcopy(ph, ad.qh[stage], g.nc);
            dcopy(pl, ad.ql[stage], g.nc);
        } else {
            WL_CK(cudaMemsetAsync(ph, 0, g.nc * sizeof(T), st));
            WL_CK(cudaMemsetAsync(pl, 0, g.nc * sizeof(T), st));
        }
        const int rc = solve(sts);
        if (stage >= 0 && ad.qwarm) {
            dcopy(ad.qh[stage], ph, g.nc);
            dcopy(ad.ql[stage], pl, g.nc);
            ad.qvalid[stage] = true;
        }
        if (Ph && dB) {
            P0("adj_param_coef", 0, g.nc);
            k_adj_param_coef<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], Ph, Pl, ph, pl, cvp(lam), w * dt,
                                                                 body_state(tt), dB[0], dB[1], S, part, ad.dpar);
            P1();
            WL_LAUNCH_CK();
            ++launches;
        }
        pmean();
        P0("adj_grad", 0, g.nc);
        k_adj_grad<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], ph, pl, S, cvp(lam), le, vvp(out), oute);
        P1();
        WL_LAUNCH_CK();
        ++launches;
        return rc;
    }

    void adj_flux(T *const (&u)[3], const T *ue, T *const (&lam)[3], T *const (&ub)[3], T *ueb) {
        P0("adj_flux", 0, g.nc);
        k_adj_flux<T, ND><<<blocks(g.nc), 256, 0, st>>>(g, cvp(u), ue, cvp(lam), vvp(ub), ueb);
        P1();
        WL_LAUNCH_CK();
        ++launches;
    }

    void adj_blend(T *const (&gin)[3], double s, T *const *ustar_b, T *const (&ub)[3], T *const (&fb)[3], double dt) {
        Vec3P<T> sb{};
        for (int a = 0; a < 3; ++a) sb.p[a] = ustar_b ? ustar_b[a] : nullptr;
        P0("adj_blend", 0, g.nc);
        k_adj_blend<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cvp(gin), (T)s, mu1n, (long long)g.nc, has_body, sb,
                                                        vvp(ub), vvp(fb), (T)dt);
        P1();
        WL_LAUNCH_CK();
        ++launches;
    }

    void adj_param_blend(T *const (&gin)[3], double s, T *const (&f)[3], const BodyTangent *dB, double tt) {
        if (user) {
            if (!vtan) return;
            P0("adj_vtan_blend", 0, g.nc);
            k_adj_vtan_blend<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cvp(gin), (T)s, mu1n, (long long)g.nc, cvp(dVt),
                                                                 S, part, ad.dpar);
            P1();
            WL_LAUNCH_CK();
            ++launches;
            return;
        }
        CVec3P<T> V{};
        for (int a = 0; a < 3; ++a) V.p[a] = Vb[a];
        P0("adj_param_blend", 0, g.nc);
        k_adj_param_blend<T, ND><<<tgrid(0), tblk(), 0, st>>>(lv[0], cvp(gin), (T)s, cvp(f), V, body_state(tt),
                                                              dB[0], dB[1], S, part, ad.dpar);
        P1();
        WL_LAUNCH_CK();
        ++launches;
    }

    // Core of the step's adjoint on device buffers. In: ad.u0 / ad.ue0 (start
    // state), ph / pl (warm start), ad.lu / ad.le (cotangents of the step's
    // velocity and exit plane), ad.lP when haveP (of its pressure). Out:
    // ad.ub / ad.ueb. With params, the heave / pitch amplitude derivative of
    // the step (and of wF . F of its pressure, wF may be null) is added into
    // ad.dpar. Leaves the velocity slots, exit planes and ph / pl changed.
    int vjp_core(double t0, double dt, bool haveP, double tol, bool params, const double *wF, wl_solve_stats *sts) {
        Range rng("wl.step_vjp");
        const size_t pb = (size_t)np * sizeof(T);
        const double t1 = t0 + dt;
        const double tol0 = cfg.tol;
        const bool gc = gq.collect, gu = gq.use;
        gq.collect = gq.use = false;
        cfg.tol = tol;
        if (has_body && (moving || body_t != t1)) body_update(t1);
        params = params && has_body;
        BodyTangent dB[2];
        if (params) { adj_alloc_params(); param_tangents(t1, dB[0], dB[1]); }
        // a sampled body's only parameter moves its velocity, not its geometry:
        // no coefficient or direct force term
        const bool geo = params && !user;
        wl_solve_stats s[2] = {};
        // forward predictor: u*, u_e* (and its blend input and pressure)
        copy_vec(vel[cur], ad.u0);
        if (g.exit_x) {
            dcopy(ueA, ad.ue0, np);
            dcopy(ueB, ad.ue0, np);
        }
        const int A0 = cur, B1 = (cur + 1) & 3, C2 = (cur + 2) & 3, D3 = (cur + 3) & 3;
        int ustar;
        if (!has_body) {
            flux<FM_PRED_U>(fargs(A0, ueB, -1, B1, dt));
            ustar = B1;
        } else {
            flux<FM_PRED_F>(fargs(A0, ueB, -1, B1, dt));
            if (params) copy_vec(ad.f1, vel[B1]);
            blend(false, B1, -1, C2);
            ustar = C2;
        }
        exit_stage(false, A0, dt);
        int r0 = project_buf(ustar, ueA, 1.0, dt, nullptr);
        copy_vec(ad.us, vel[ustar]);
        if (g.exit_x) dcopy(ad.ues, ueA, np);
        int r0c = WL_OK;
        if (params) {
            // forward corrector: its blend input and pressure
            dcopy(ad.P1h, ph, g.nc);
            dcopy(ad.P1l, pl, g.nc);
            flux<FM_CORR_F>(fargs(ustar, ueA, A0, B1, dt));
            copy_vec(ad.f2, vel[B1]);
            blend(true, B1, ustar, D3);
            exit_stage(true, ustar, dt);
            r0c = project_buf(D3, ueA, 0.5, dt, nullptr);
            dcopy(ad.P2h, ph, g.nc);
            dcopy(ad.P2l, pl, g.nc);
            if (wF && geo) {
                // direct dependence of wF . F on the body at fixed pressure
                pmean();
                P0("force_dparam", 0, g.nc);
                k_force_dparam<T><<<blocks(g.nc), 256, 0, st>>>(g, body_state(t1), dB[0], dB[1], ph, pl, lv[0].invD,
                                                                wF[0], wF[1], wF[2], S, part, ad.dpar);
                P1();
                WL_LAUNCH_CK();
                ++launches;
            }
        }
        // reverse: corrector projection, exit, blend, flux at u*
        int r1 = proj_vjp(ad.lu, g.exit_x ? ad.le : nullptr, haveP ? ad.lP : nullptr, 0.5, dt, ad.x, ad.xe, &s[1],
                          geo ? ad.P2h : nullptr, geo ? ad.P2l : nullptr, geo ? dB : nullptr, t1, 1);
        zero_vec(ad.ub);
        zero_vec(ad.usb);
        if (g.exit_x) {
            WL_CK(cudaMemsetAsync(ad.ueb, 0, pb, st));
            WL_CK(cudaMemsetAsync(ad.uesb, 0, pb, st));
            k_adj_exit<T, true><<<1, 1024, 0, st>>>(g, ad.xe, (T)dt, ad.ueb, ad.uesb, ad.usb[0]);
            WL_LAUNCH_CK();
            ++launches;
        }
        if (params) adj_param_blend(ad.x, 0.5, ad.f2, dB, t1);
        adj_blend(ad.x, 0.5, ad.usb, ad.ub, ad.fb, dt);
        adj_flux(ad.us, ad.ues, ad.fb, ad.usb, ad.uesb);
        // predictor projection, exit, blend, flux at u0
        int r2 = proj_vjp(ad.usb, g.exit_x ? ad.uesb : nullptr, nullptr, 1.0, dt, ad.x, ad.xe, &s[0],
                          geo ? ad.P1h : nullptr, geo ? ad.P1l : nullptr, geo ? dB : nullptr, t1, 0);
        if (g.exit_x) {
            k_adj_exit<T, false><<<1, 1024, 0, st>>>(g, ad.xe, (T)dt, ad.ueb, ad.ueb, ad.ub[0]);
            WL_LAUNCH_CK();
            ++launches;
        }
        if (params) adj_param_blend(ad.x, 1.0, ad.f1, dB, t1);
        adj_blend(ad.x, 1.0, nullptr, ad.ub, ad.fb, dt);
        adj_flux(ad.u0, ad.ue0, ad.fb, ad.ub, ad.ueb);
        cfg.tol = tol0;
        gq.collect = gc;
        gq.use = gu;
        if (sts) { sts[0] = s[0]; sts[1] = s[1]; }
        int rc = WL_OK;
        for (int r : {r0, r0c, r1, r2})
            if (r != WL_OK && rc == WL_OK) rc = r;
        if (rc == WL_ERR_NONFINITE) err = "non-finite values in the adjoint step";
        else if (rc == WL_ERR_NOT_CONVERGED) err = "a Poisson solve of the adjoint step did not reach tol";
        return rc;
    }

    void backup_state() {
        copy_vec(ad.bku, vel[cur]);
        dcopy(ad.bkue, ueA, np);
        dcopy(ad.bkph, ph, g.nc);
        dcopy(ad.bkpl, pl, g.nc);
    }
    void restore_state(double body_t0) {
        copy_vec(vel[cur], ad.bku);
        dcopy(ueA, ad.bkue, np);
        dcopy(ph, ad.bkph, g.nc);
        dcopy(pl, ad.bkpl, g.nc);
        if (has_body && body_t != body_t0 && body_t0 >= 0) body_update(body_t0);
    }

    // Vector-Jacobian product of one step (mom_step with a fixed dt, body
    // measured at t0 + dt) at the start state (u0, ue0), warm start P0: given
    // the cotangents (lu, le) of the step's velocity and exit plane and lP of
    // its reported pressure, returns (ub, ueb) for (u0, ue0). The sim's state
    // (velocity, exit plane, pressure, time, body) is left as it was.
    int step_vjp(double t0, double dt, const void *u0, const void *ue0, const double *P0in, const void *lu,
                 const void *le, const double *lP, double tol, void *ub, void *ueb, wl_solve_stats *sts) override {
        if (!(dt > 0)) throw Err{WL_ERR_ARG, "step_vjp: dt must be positive"};
        adj_alloc();
        const size_t vb = g.nc * sizeof(T), pb = (size_t)np * sizeof(T);
        const double body_t0 = body_t;
        backup_state();
        for (int a = 0; a < g.ndim; ++a) {
            WL_CK(cudaMemcpyAsync(ad.u0[a], (const char *)u0 + a * vb, vb, cudaMemcpyDefault, st));
            WL_CK(cudaMemcpyAsync(ad.lu[a], (const char *)lu + a * vb, vb, cudaMemcpyDefault, st));
        }
        if (g.exit_x) {
            if (ue0) WL_CK(cudaMemcpyAsync(ad.ue0, ue0, pb, cudaMemcpyDefault, st));
            else k_fill<T><<<blocks(np), 256, 0, st>>>((long long)np, (T)g.U[0], ad.ue0);
            if (le) WL_CK(cudaMemcpyAsync(ad.le, le, pb, cudaMemcpyDefault, st));
            else WL_CK(cudaMemsetAsync(ad.le, 0, pb, st));
        }
        if (lP) WL_CK(cudaMemcpyAsync(ad.lP, lP, g.nc * sizeof(double), cudaMemcpyDefault, st));
        if (P0in) {
            WL_CK(cudaMemcpyAsync(pout, P0in, g.nc * sizeof(double), cudaMemcpyDefault, st));
            k_pin<T><<<blocks(g.nc), 256, 0, st>>>(g, pout, ph, pl);
            WL_LAUNCH_CK();
            ++launches;
        } else {
            WL_CK(cudaMemsetAsync(ph, 0, vb, st));
            WL_CK(cudaMemsetAsync(pl, 0, vb, st));
        }
        const int rc = vjp_core(t0, dt, lP != nullptr, tol, false, nullptr, sts);
        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemcpyAsync((char *)ub + a * vb, ad.ub[a], vb, cudaMemcpyDefault, st));
        if (ueb && g.exit_x) WL_CK(cudaMemcpyAsync(ueb, ad.ueb, pb, cudaMemcpyDefault, st));
        restore_state(body_t0);
        WL_CK(cudaStreamSynchronize(st));
        prof.flush();
        return rc;
    }

    // Weighted pressure derivative of the force into ad.lP: scale * sum_a w_a dF_a/dp.
    void force_dp_w(double tt, const double *w, double scale) {
        adj_alloc();
        if (!has_body) {
            WL_CK(cudaMemsetAsync(ad.lP, 0, g.nc * sizeof(double), st));
            return;
        }
        with_centre(tt, [&](auto cs) {
            k_force_dp<T, decltype(cs)><<<blocks(g.nc), 256, 0, st>>>(g, cs, lv[0].invD, w[0] * scale, w[1] * scale,
                                                                      w[2] * scale, ad.lP);
        });
        WL_LAUNCH_CK();
        ++launches;
    }

    void force_dp(int axis, double scale, double *gout) override {
        if (axis < 0 || axis >= g.ndim) throw Err{WL_ERR_ARG, "force_dp: axis out of range"};
        double w[3] = {0, 0, 0};
        w[axis] = 1.0;
        force_dp_w(body_t, w, scale);
        WL_CK(cudaMemcpyAsync(gout, ad.lP, g.nc * sizeof(double), cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    // ------------------------------------------------- checkpointed window
    Snap snap_alloc() {
        Snap s{};
        for (int a = 0; a < g.ndim; ++a) s.u[a] = alloc_n<T>(g.nc);
        s.ue = alloc_n<T>(np);
        s.ph = alloc_n<T>(g.nc);
        s.pl = alloc_n<T>(g.nc);
        return s;
    }
    void snap_take(Snap &s) {
        copy_vec(s.u, vel[cur]);
        dcopy(s.ue, ueA, np);
        dcopy(s.ph, ph, g.nc);
        dcopy(s.pl, pl, g.nc);
        s.t = t;
    }
    void snap_put(const Snap &s) {
        copy_vec(vel[cur], s.u);
        dcopy(ueA, s.ue, np);
        dcopy(ph, s.ph, g.nc);
        dcopy(pl, s.pl, g.nc);
        t = s.t;
    }

    int window_forward(int nsteps, int ckpt, const double *dts, const double *w, const double *step_w, int viscous,
                       double *J, double *dts_out) override {
        if (nsteps < 1 || ckpt < 1) throw Err{WL_ERR_ARG, "window: nsteps and ckpt_every must be >= 1"};
        adj_alloc();
        const int nck = (nsteps + ckpt - 1) / ckpt;
        if ((int)win.ck.size() < nck) while ((int)win.ck.size() < nck) win.ck.push_back(snap_alloc());
        if ((int)win.seg.size() < ckpt) while ((int)win.seg.size() < ckpt) win.seg.push_back(snap_alloc());
        if (!win.fin.ue) win.fin = snap_alloc();
        win.active = false;
        // the learned guesses change the converged fields only within the
        // solver tolerance, but the backward sweep's recomputation must repeat
        // this forward run exactly: both stay off over the window
        const bool tgu = tg.use, gqu = gq.use;
        tg.use = gq.use = false;
        struct Restore { bool &a, &b; bool va, vb; ~Restore() { a = va; b = vb; } } rs{tg.use, gq.use, tgu, gqu};
        win.n = nsteps;
        win.k = ckpt;
        for (int a = 0; a < 3; ++a) win.w[a] = w ? w[a] : 0.0;
        win.dts.assign(nsteps, 0.0);
        win.ws.assign(nsteps, 1.0);
        win.visc = viscous != 0;
        if (step_w) for (int n = 0; n < nsteps; ++n) win.ws[n] = step_w[n];
        double Jv = 0.0;
        for (int n = 0; n < nsteps; ++n) {
            if (n % ckpt == 0) snap_take(win.ck[n / ckpt]);
            const double dt = dts ? dts[n] : dt_next;
            win.dts[n] = dt;
            const int rc = mom_step(dt, nullptr);
            if (rc != WL_OK) return rc;
            if (w && has_body && win.ws[n] != 0.0) {
                double F[3];
                forces(F);
                if (win.visc) {
                    double Fv[3];
                    forces_viscous(Fv);
                    for (int a = 0; a < 3; ++a) F[a] += Fv[a];
                }
                Jv += win.ws[n] * (w[0] * F[0] + w[1] * F[1] + w[2] * F[2]);
            }
        }
        snap_take(win.fin);
        win.fin_dt_next = dt_next;
        WL_CK(cudaStreamSynchronize(st));
        if (J) *J = Jv;
        if (dts_out) for (int n = 0; n < nsteps; ++n) dts_out[n] = win.dts[n];
        win.active = true;
        return WL_OK;
    }

    int window_backward(double gJ, const void *luf, const void *lef, double tol, void *du0, void *due0,
                        double *dparams) override {
        if (!win.active) throw Err{WL_ERR_STATE, "window_backward: no forward window is held"};
        adj_alloc();
        const size_t vb = g.nc * sizeof(T), pb = (size_t)np * sizeof(T);
        const bool params = dparams != nullptr && has_body;
        const bool force = has_body && (win.w[0] != 0 || win.w[1] != 0 || win.w[2] != 0) && gJ != 0.0;

        // final cotangents
        for (int a = 0; a < g.ndim; ++a) {
            if (luf) WL_CK(cudaMemcpyAsync(ad.lu[a], (const char *)luf + a * vb, vb, cudaMemcpyDefault, st));
            else WL_CK(cudaMemsetAsync(ad.lu[a], 0, vb, st));
        }
        if (g.exit_x) {
            if (lef) WL_CK(cudaMemcpyAsync(ad.le, lef, pb, cudaMemcpyDefault, st));
            else WL_CK(cudaMemsetAsync(ad.le, 0, pb, st));
        }
        WL_CK(cudaMemsetAsync(ad.dpar, 0, 2 * sizeof(double), st));
        win.solves = win.unconverged = win.max_vc = 0;
        win.worst_step = -1;
        win.max_rel = 0.0;
        const bool tgu = tg.use, gqu = gq.use;
        tg.use = gq.use = false;
        struct Restore { bool &a, &b; bool va, vb; ~Restore() { a = va; b = vb; } } rs{tg.use, gq.use, tgu, gqu};
        ad.qwarm = true;
        ad.qvalid[0] = ad.qvalid[1] = false;
        struct QOff { bool &q; ~QOff() { q = false; } } qoff{ad.qwarm};
        // the viscous force is linear in the velocity: its gradient is one
        // field for the window (the body is fixed or moves the same in every
        // recomputation), added to the velocity cotangent after each step
        const bool visc = force && win.visc;
        if (visc) {
            for (int a = 0; a < g.ndim; ++a) {
                if (!win.gv[a]) win.gv[a] = alloc_n<T>(g.nc);
                WL_CK(cudaMemsetAsync(win.gv[a], 0, vb, st));
            }
            if (!win.gve) win.gve = alloc_n<T>(np);
            WL_CK(cudaMemsetAsync(win.gve, 0, pb, st));
        }
        double visc_t = -1.0;
        int rc = WL_OK;
        const int nseg = (win.n + win.k - 1) / win.k;
        for (int sgi = nseg - 1; sgi >= 0 && rc == WL_OK; --sgi) {
            const int n0 = sgi * win.k, n1 = std::min(win.n, n0 + win.k);
            // recompute the segment's start states from its checkpoint
            snap_put(win.ck[sgi]);
            for (int n = n0; n < n1; ++n) {
                snap_take(win.seg[n - n0]);
                if (n + 1 < n1) {
                    const int r = mom_step(win.dts[n], nullptr);
                    if (r != WL_OK && r != WL_ERR_NOT_CONVERGED) { rc = r; break; }
                }
            }
            for (int n = n1 - 1; n >= n0 && rc == WL_OK; --n) {
                const Snap &s = win.seg[n - n0];
                const double dt = win.dts[n];
                copy_vec(ad.u0, s.u);
                dcopy(ad.ue0, s.ue, np);
                dcopy(ph, s.ph, g.nc);
                dcopy(pl, s.pl, g.nc);
                if (has_body && (moving || body_t != s.t + dt)) body_update(s.t + dt);
                const double gn = gJ * win.ws[n];
                const bool fn = force && gn != 0.0;
                const double wF[3] = {gn * win.w[0], gn * win.w[1], gn * win.w[2]};
                if (fn) force_dp_w(s.t + dt, win.w, gn);
                if (fn && visc) {
                    if (visc_t != body_t || moving) {
                        // (re)form d(w . F_v)/du for the body as measured now
                        for (int a = 0; a < g.ndim; ++a) WL_CK(cudaMemsetAsync(win.gv[a], 0, vb, st));
                        WL_CK(cudaMemsetAsync(win.gve, 0, pb, st));
                        with_centre(body_t, [&](auto cs) {
                            k_force_visc_du<T, decltype(cs)><<<blocks(g.nc), 256, 0, st>>>(
                                g, cs, win.w[0], win.w[1], win.w[2], 1.0, vvp(win.gv), g.exit_x ? win.gve : nullptr);
                        });
                        WL_LAUNCH_CK();
                        ++launches;
                        visc_t = body_t;
                    }
                    for (int a = 0; a < g.ndim; ++a)
                        k_axpy<T><<<blocks(g.nc), 256, 0, st>>>((long long)g.nc, (T)gn, win.gv[a], ad.lu[a]);
                    if (g.exit_x) k_axpy<T><<<blocks(np), 256, 0, st>>>((long long)np, (T)gn, win.gve, ad.le);
                    WL_LAUNCH_CK();
                    launches += g.ndim + (g.exit_x ? 1 : 0);
                }
                wl_solve_stats ss[2] = {};
                const int r = vjp_core(s.t, dt, fn, tol, params, fn ? wF : nullptr, ss);
                for (const wl_solve_stats &q : ss) {
                    ++win.solves;
                    if (q.rel_resid > tol) ++win.unconverged;
                    win.max_vc = std::max(win.max_vc, q.vcycles);
                    if (q.rel_resid > win.max_rel) { win.max_rel = q.rel_resid; win.worst_step = n; }
                }
                if (r == WL_ERR_NONFINITE) rc = r;
                for (int a = 0; a < 3; ++a) std::swap(ad.lu[a], ad.ub[a]);
                std::swap(ad.le, ad.ueb);
            }
        }
        if (rc == WL_OK) {
            for (int a = 0; a < g.ndim; ++a)
                if (du0) WL_CK(cudaMemcpyAsync((char *)du0 + a * vb, ad.lu[a], vb, cudaMemcpyDefault, st));
            if (due0 && g.exit_x) WL_CK(cudaMemcpyAsync(due0, ad.le, pb, cudaMemcpyDefault, st));
            if (dparams) WL_CK(cudaMemcpyAsync(dparams, ad.dpar, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        // back to the state after the window
        snap_put(win.fin);
        dt_next = win.fin_dt_next;
        if (has_body && (moving || body_t != t)) body_update(t);
        WL_CK(cudaStreamSynchronize(st));
        prof.flush();
        return rc;
    }

    // ------------------------------------------------- checkpoint / resume
    struct StateHeader {
        char magic[8];
        int version, ndim, n[3], precision, body_kind, pad;
        double t, dt_next, body_t;
    };
    size_t state_bytes() const {
        return sizeof(StateHeader) + ((size_t)ND * g.nc + (size_t)np + 2 * (size_t)g.nc) * sizeof(T);
    }
    void state_size(size_t *bytes) override { *bytes = state_bytes(); }

    void get_state(void *buf, size_t bytes) override {
        if (bytes < state_bytes()) throw Err{WL_ERR_ARG, "get_state: buffer smaller than wl_state_size"};
        StateHeader h{};
        std::memcpy(h.magic, "WLSTATE", 8);
        h.version = 1;
        h.ndim = ND;
        for (int a = 0; a < 3; ++a) h.n[a] = g.n[a];
        h.precision = cfg.precision;
        h.body_kind = body.kind;
        h.t = t;
        h.dt_next = dt_next;
        h.body_t = body_t;
        char *o = (char *)buf;
        WL_CK(cudaMemcpyAsync(o, &h, sizeof(h), cudaMemcpyDefault, st));
        size_t off = sizeof(h);
        const size_t vb = g.nc * sizeof(T);
        for (int a = 0; a < ND; ++a, off += vb) WL_CK(cudaMemcpyAsync(o + off, vel[cur][a], vb, cudaMemcpyDefault, st));
        WL_CK(cudaMemcpyAsync(o + off, ueA, (size_t)np * sizeof(T), cudaMemcpyDefault, st));
        off += (size_t)np * sizeof(T);
        WL_CK(cudaMemcpyAsync(o + off, ph, vb, cudaMemcpyDefault, st));
        WL_CK(cudaMemcpyAsync(o + off + vb, pl, vb, cudaMemcpyDefault, st));
        WL_CK(cudaStreamSynchronize(st));
    }

    void set_state(const void *buf, size_t bytes) override {
        if (bytes < state_bytes()) throw Err{WL_ERR_ARG, "set_state: buffer smaller than wl_state_size"};
        StateHeader h{};
        WL_CK(cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDefault));
        bool same = std::memcmp(h.magic, "WLSTATE", 8) == 0 && h.version == 1 && h.ndim == ND &&
                    h.precision == cfg.precision && h.body_kind == body.kind;
        for (int a = 0; a < 3; ++a) same = same && h.n[a] == g.n[a];
        if (!same) throw Err{WL_ERR_ARG, "set_state: the state was taken from a sim of another grid, precision or body kind"};
        const char *o = (const char *)buf;
        size_t off = sizeof(h);
        const size_t vb = g.nc * sizeof(T);
        for (int a = 0; a < ND; ++a, off += vb) WL_CK(cudaMemcpyAsync(vel[cur][a], o + off, vb, cudaMemcpyDefault, st));
        WL_CK(cudaMemcpyAsync(ueA, o + off, (size_t)np * sizeof(T), cudaMemcpyDefault, st));
        off += (size_t)np * sizeof(T);
        WL_CK(cudaMemcpyAsync(ph, o + off, vb, cudaMemcpyDefault, st));
        WL_CK(cudaMemcpyAsync(pl, o + off + vb, vb, cudaMemcpyDefault, st));
        t = h.t;
        dt_next = h.dt_next;
        win.active = false;
        // a measured body at the time it stood for: the coefficients of a full
        // measure equal those a run of box measures left (outside a box only
        // the body velocity, which no kernel reads there, may differ)
        if (has_body && !user && h.body_t >= 0) measure_body(h.body_t, false);
        else body_t = h.body_t;
        WL_CK(cudaStreamSynchronize(st));
    }

    void window_stats(int *out4, double *max_rel) override {
        if (out4) { out4[0] = win.solves; out4[1] = win.unconverged; out4[2] = win.max_vc; out4[3] = win.worst_step; }
        if (max_rel) *max_rel = win.max_rel;
    }

    void set_body(const wl_body *bd) override {
        if (!bd || bd->kind != body.kind) throw Err{WL_ERR_ARG, "set_body: the body kind cannot change"};
        body = *bd;
        moving = has_body && !user && (body.heave_amp != 0.0 || body.pitch_amp != 0.0);
        win.active = false;
        if (has_body) body_update(body_t >= 0 ? body_t : t);
        // the coarsest level's dense operator follows the new coefficients
        const bool want = gl[nlev - 1].nc <= dense_max;
        const bool was = cdense;
        cdense = want && coarse_dense();
        if (cdense != was) build_vcycle_graph();
        WL_CK(cudaStreamSynchronize(st));
    }

    // Largest coarsest level (cells) that the dense solution operator solves
    // (0 to WL_DENSE_MAX; 256 at creation); a larger one is solved by the
    // one-block PCG. Ends an open adjoint window (its solves would change).
    void set_coarse_dense_max(int m) override {
        if (m < 0 || m > WL_DENSE_MAX) throw Err{WL_ERR_ARG, "set_coarse_dense_max: max_cells must lie in [0, 1024]"};
        dense_max = m;
        win.active = false;
        const bool was = cdense;
        cdense = gl[nlev - 1].nc <= dense_max && coarse_dense();
        if (cdense != was) build_vcycle_graph();
        WL_CK(cudaStreamSynchronize(st));
    }

    void info(int *levels, long long *nl) override {
        if (levels) *levels = nlev;
        if (nl) *nl = launches;
    }
};

}  // namespace wl
