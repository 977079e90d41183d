// k_adjoint.cuh -- transposed kernels of one time step (vector-Jacobian
// products), for the hand-written reverse-mode adjoint of the step.
//
// The step (Sec. 2: explicit predictor-corrector, BDIM blend, projection) is
// piecewise linear-quadratic in the velocity; its Jacobian at a point is taken
// with the flux limiter's branches frozen there (a subgradient at ties, with
// the tie rule of median_w below). Transposes:
//   R^T  the convection-diffusion flux (Sec. 2 F-dot, flux-limited QUICK):
//        every face flux F scatters mu_F * dF/d(sample) to the six velocity
//        samples it reads, mu_F = lam_a[I] - lam_a[I - e_b];
//   B^T  the BDIM blend u = V + mu0 (f - V) + mu1 n.grad(f - V): gathered;
//   P^T  the projection u - w dt c grad A^+ div u / (w dt): symmetric A, so the
//        adjoint reuses the same multigrid solve on div(c lam);
//   E^T  the convective exit with its uniform mass correction.
#pragma once
#include "wl_common.cuh"
#include "k_poisson.cuh"
#include "k_body.cuh"

// Storage of velocity sample (a, i, j, k) under the boundary rule of
// vel_sample: a pointer into the component array or the exit plane, or null
// for a constant (U_a on a non-periodic upper boundary face).
template <typename T>
__device__ __forceinline__ T *vel_slot(const GridD &g, T *ua, T *ue, int a, int i, int j, int k) {
    int I[3] = {i, j, k};
    bool up = false;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax >= g.ndim) { I[ax] = 0; continue; }
        const int N = g.n[ax];
        if (g.per[ax]) {
            I[ax] = wrapi(I[ax], N);
        } else if (ax == a) {
            if (I[ax] < 0) I[ax] = 0;
            else if (I[ax] >= N) { I[ax] = N; up = true; }
        } else {
            I[ax] = I[ax] < 0 ? 0 : (I[ax] > N - 1 ? N - 1 : I[ax]);
        }
    }
    if (up) return (a == 0 && g.exit_x) ? ue + (I[1] + (long long)g.n[1] * I[2]) : nullptr;
    return ua + lin3(g, I[0], I[1], I[2]);
}

// Median of three and which argument (0, 1, 2) it is. Tie rule: m1 = min(a, b)
// is a when a <= b, the upper value M1 is b then; m2 = min(M1, c) is M1 when
// M1 <= c; the result is m1 when m1 >= m2, else m2.
template <typename T>
__device__ __forceinline__ T median_w(T a, T b, T c, int &w) {
    const bool ab = a <= b;
    const T m1 = ab ? a : b, M1 = ab ? b : a;
    const int w1 = ab ? 0 : 1, wM = ab ? 1 : 0;
    const bool mc = M1 <= c;
    const T m2 = mc ? M1 : c;
    const int w2 = mc ? wM : 2;
    if (m1 >= m2) { w = w1; return m1; }
    w = w2;
    return m2;
}

// Limited QUICK value (5c + 2d - uu)/6 bounded by median(phi, c, median(10c -
// 9uu, c, d)) and its partial derivatives (duu, dc, dd) on the active branch.
template <typename T>
__device__ __forceinline__ T quick_grad(T uu, T c, T d, T &guu, T &gc, T &gd) {
    const T phi = (T(5) * c + T(2) * d - uu) * T(1.0 / 6.0);
    int wi, wo;
    const T inner = median_w(T(10) * c - T(9) * uu, c, d, wi);
    const T val = median_w(phi, c, inner, wo);
    guu = T(0); gc = T(0); gd = T(0);
    if (wo == 0) { guu = T(-1.0 / 6.0); gc = T(5.0 / 6.0); gd = T(2.0 / 6.0); }
    else if (wo == 1) gc = T(1);
    else if (wi == 0) { guu = T(-9); gc = T(10); }
    else if (wi == 1) gc = T(1);
    else gd = T(1);
    return val;
}

template <typename T>
__device__ __forceinline__ void add_to(T *p, T v) {
    if (p && v != T(0)) atomicAdd(p, v);
}

// Cotangent of the flux of u_a along b through the lower b-face at position I
// (I[b] in 0..N_b on a non-periodic axis b): rows I and I - e_b of r_a, with
// r_a zero on the lower boundary face of a non-periodic axis a.
template <typename T>
__device__ __forceinline__ T flux_cot(const GridD &g, const T *lam, int a, int b, const int (&I)[3]) {
    const int N = g.n[b];
    T m = T(0);
    int J[3] = {I[0], I[1], I[2]};
    auto row = [&](const int (&K)[3]) -> T {
        if (!g.per[a] && K[a] == 0) return T(0);
        return lam[lin3(g, K[0], K[1], K[2])];
    };
    if (g.per[b]) {
        J[b] = wrapi(I[b], N);
        m += row(J);
        J[b] = wrapi(I[b] - 1, N);
        m -= row(J);
    } else {
        if (I[b] <= N - 1) m += row(J);
        if (I[b] >= 1) { J[b] = I[b] - 1; m -= row(J); }
    }
    return m;
}

// Scatter mu * dF/d(samples) of the flux of u_a along b at face position I.
template <typename T>
__device__ __forceinline__ void flux_vjp_face(const GridD &g, CVec3P<T> u, const T *ue, Vec3P<T> ub, T *ueb, int a,
                                              int b, const int (&I)[3], T mu) {
    if (mu == T(0)) return;
    int db[3] = {0, 0, 0}, da[3] = {0, 0, 0};
    db[b] = 1;
    da[a] = 1;
    const T nu = (T)g.nu;
    // samples: u_b at I and I - e_a; u_a at I - 2e_b, I - e_b, I, I + e_b
    const T vb0 = vel_sample<T>(g, u.p[b], ue, b, I[0], I[1], I[2]);
    const T vb1 = vel_sample<T>(g, u.p[b], ue, b, I[0] - da[0], I[1] - da[1], I[2] - da[2]);
    const T sm2 = vel_sample<T>(g, u.p[a], ue, a, I[0] - 2 * db[0], I[1] - 2 * db[1], I[2] - 2 * db[2]);
    const T sm1 = vel_sample<T>(g, u.p[a], ue, a, I[0] - db[0], I[1] - db[1], I[2] - db[2]);
    const T s0 = vel_sample<T>(g, u.p[a], ue, a, I[0], I[1], I[2]);
    const T sp1 = vel_sample<T>(g, u.p[a], ue, a, I[0] + db[0], I[1] + db[1], I[2] + db[2]);
    const T Uf = T(0.5) * (vb0 + vb1);
    T guu, gc, gd, phi;
    const bool pos = Uf > T(0);
    if (pos) phi = quick_grad<T>(sm2, sm1, s0, guu, gc, gd);
    else phi = quick_grad<T>(sp1, s0, sm1, guu, gc, gd);
    const T hb = mu * T(0.5) * phi;
    add_to(vel_slot<T>(g, ub.p[b], ueb, b, I[0], I[1], I[2]), hb);
    add_to(vel_slot<T>(g, ub.p[b], ueb, b, I[0] - da[0], I[1] - da[1], I[2] - da[2]), hb);
    T *pm2 = vel_slot<T>(g, ub.p[a], ueb, a, I[0] - 2 * db[0], I[1] - 2 * db[1], I[2] - 2 * db[2]);
    T *pm1 = vel_slot<T>(g, ub.p[a], ueb, a, I[0] - db[0], I[1] - db[1], I[2] - db[2]);
    T *p0 = vel_slot<T>(g, ub.p[a], ueb, a, I[0], I[1], I[2]);
    T *pp1 = vel_slot<T>(g, ub.p[a], ueb, a, I[0] + db[0], I[1] + db[1], I[2] + db[2]);
    const T mU = mu * Uf;
    if (pos) {
        add_to(pm2, mU * guu);
        add_to(pm1, mU * gc + mu * nu);
        add_to(p0, mU * gd - mu * nu);
    } else {
        add_to(pp1, mU * guu);
        add_to(p0, mU * gc - mu * nu);
        add_to(pm1, mU * gd + mu * nu);
    }
}

// (ub, ueb) += J_R(u, ue)^T lam. One thread per cell owns the fluxes at its
// lower faces, and on a non-periodic upper domain edge also the boundary flux
// one face further; contributions land by atomic adds (order-dependent in the
// last bit only).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_flux(GridD g, CVec3P<T> u, const T *ue, CVec3P<T> lam, Vec3P<T> ub,
                                                  T *ueb) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
#pragma unroll
            for (int b = 0; b < NDIM; ++b) {
                const int I[3] = {i, j, k};
                flux_vjp_face<T>(g, u, ue, ub, ueb, a, b, I, flux_cot<T>(g, lam.p[a], a, b, I));
                const int Ib[3] = {i, j, k};
                if (!g.per[b] && Ib[b] == g.n[b] - 1) {
                    int J[3] = {i, j, k};
                    J[b] += 1;
                    flux_vjp_face<T>(g, u, ue, ub, ueb, a, b, J, flux_cot<T>(g, lam.p[a], a, b, J));
                }
            }
    }
}

// Blend transposed (gathered). gin is the cotangent of the blended velocity;
// it is masked to zero on lower boundary faces of non-periodic axes (their
// value is the constant U_a) and scaled by s (1/2 in the corrector, whose
// blend is averaged with u*). Then
//   ustar_b += s gin            (corrector only, ustar_b may be null)
//   ub      += B^T (s gin)      (the start velocity enters f = u0 + dt r)
//   fb       = dt B^T (s gin)   (cotangent of r, for the flux transpose)
// B^T g on face a at J: mu0 g[J] + sum_b 1/2 m_ab[I] g[I] over the I whose
// clamped / wrapped upper neighbour along b is J, minus the same over the I
// whose lower neighbour is J. Tiles whose coefficients are uniform carry no
// body term (mu0 = 1, mu1 = 0 there and in their one-cell halo).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_blend(LevelD<T> L, CVec3P<T> gin, T s, const T *mu1n0, long long mstride,
                                                   bool body, Vec3P<T> ustar_b, Vec3P<T> ub, Vec3P<T> fb, T dt) {
    const GridD &g = L.g;
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        const int J[3] = {i, j, k};
        auto gm = [&](int a, const int (&K)[3]) -> T {
            if (!g.per[a] && K[a] == 0) return T(0);
            return s * gin.p[a][lin3(g, K[0], K[1], K[2])];
        };
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const T gj = gm(a, J);
            if (ustar_b.p[a]) ustar_b.p[a][idx] += gj;
            T v;
            if (!body || uni) {
                v = gj;
            } else {
                v = L.c[a][idx] * gj;
#pragma unroll
                for (int b = 0; b < NDIM; ++b) {
                    const int N = g.n[b];
                    const T *m = mu1n0 + (long long)(a * 3 + b) * mstride;
                    // I = J - e_b has upper neighbour J; at the top edge J itself too
                    int K[3] = {J[0], J[1], J[2]};
                    if (g.per[b]) {
                        K[b] = wrapi(J[b] - 1, N);
                        v += T(0.5) * m[lin3(g, K[0], K[1], K[2])] * gm(a, K);
                        K[b] = wrapi(J[b] + 1, N);
                        v -= T(0.5) * m[lin3(g, K[0], K[1], K[2])] * gm(a, K);
                    } else {
                        if (J[b] >= 1) { K[b] = J[b] - 1; v += T(0.5) * m[lin3(g, K[0], K[1], K[2])] * gm(a, K); }
                        if (J[b] == N - 1) v += T(0.5) * m[idx] * gj;
                        if (J[b] <= N - 2) { K[b] = J[b] + 1; v -= T(0.5) * m[lin3(g, K[0], K[1], K[2])] * gm(a, K); }
                        if (J[b] == 0) v -= T(0.5) * m[idx] * gj;
                    }
                }
            }
            ub.p[a][idx] += v;
            fb.p[a][idx] = dt * v;
        }
    });
}

// Right-hand side of the projection's adjoint solve: b = div(c lam) + lP/(w dt),
// with c = 0 on the upper boundary faces of non-periodic axes (the exit plane
// carries no Poisson coefficient). bl (the low half of the pair) is zeroed.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_rhs(LevelD<T> L, CVec3P<T> lam, const double *lP, double inv_wdt, T *b,
                                                 T *bl) {
    const GridD &g = L.g;
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, uni, i, j, k, idx, ip, im, cp, cm);
        T s = T(0);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            if (cp[a] != T(0)) s += cp[a] * lam.p[a][ip[a]];
            s -= cm[a] * lam.p[a][idx];
        }
        if (lP) s += (T)(lP[idx] * inv_wdt);
        b[idx] = s;
        bl[idx] = T(0);
    });
}

// Projection transposed, final step: ub = lam + D^T q, with q = ph + pl - mean
// over active rows (0 on inactive rows); the exit plane's cotangent gains q of
// the last cell row (the exit face enters the divergence of that cell).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_grad(LevelD<T> L, const T *ph, const T *pl, const DevScalars *S,
                                                  CVec3P<T> lam, const T *le, Vec3P<T> ub, T *ueb) {
    const GridD &g = L.g;
    const double pm = S->pmean;
    const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    auto qv = [&](long long id) -> T {
        return L.invD[id] != T(0) ? (T)(((double)ph[id] - pm) + (double)pl[id]) : T(0);
    };
    for_cells<NDIM>(g, L.tl, nullptr, [&](int i, int j, int k, long long idx, bool) {
        const int I[3] = {i, j, k};
        const T q0 = qv(idx);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            T qm = T(0);
            if (I[a] > 0) qm = qv(idx - st[a]);
            else if (g.per[a]) qm = qv(idx + (long long)(g.n[a] - 1) * st[a]);
            ub.p[a][idx] = lam.p[a][idx] + (qm - q0);
        }
        if (g.exit_x && i == g.n[0] - 1) {
            const long long p = j + (long long)g.n[1] * k;
            ueb[p] = (le ? le[p] : T(0)) + q0;
        }
    });
}

// Exit condition transposed (one block). ein is the cotangent of the exit plane
// after the stage; its mean is removed (the uniform mass correction), then
//   ue0_b += w e;  ueG_b -= w dt U e;  uG_b[last x face] += w dt U e,
// and in the corrector (w = 1/2), where ueG is the star plane u_e* that the
// stage also averages with, ueG_b += e/2. ue0b and ueGb may alias (predictor).
template <typename T, bool CORR>
__global__ void k_adj_exit(GridD g, const T *ein, T dt, T *ue0b, T *ueGb, T *uGxb) {
    const int np = g.n[1] * (g.ndim == 3 ? g.n[2] : 1);
    const int n0 = g.n[0];
    __shared__ double sh[32];
    T acc[1] = {T(0)};
    double out[1];
    for (int p = threadIdx.x; p < np; p += blockDim.x) acc[0] += ein[p];
    block_reduce<1, false, T>(acc, out, sh);
    if (threadIdx.x == 0) sh[0] = out[0];
    __syncthreads();
    const T m = (T)(sh[0] / (double)np);
    const T w = CORR ? T(0.5) : T(1);
    const T Ub = (T)g.U[0];
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const T e = ein[p] - m;
        ue0b[p] += w * e;
        ueGb[p] += (CORR ? T(0.5) * e : T(0)) - w * dt * Ub * e;
        uGxb[(long long)(n0 - 1) + (long long)n0 * p] += w * dt * Ub * e;
    }
}

// Pressure derivative of the weighted force w . F on the body:
// F = -sum_I (p_I - mean) n(x_I) K_eps(d(x_I)) over active cells, so
// d(w.F)/dp_I = -(w . n) K on active cells of the kernel band (the mean's share
// is removed by the adjoint solve, whose right-hand side is made mean-free).
template <typename T, typename CS>
__global__ void k_force_dp(GridD g, CS cs, const T *invD, double w0, double w1, double w2, double *out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        double v = 0.0, K, nd[3];
        if (invD[idx] != T(0) && cs.template eval<T>(g, i, j, k, idx, K, nd))
            v = -(w0 * nd[0] + w1 * nd[1] + w2 * nd[2]) * K;
        out[idx] = v;
    }
}

// Velocity derivative of the weighted viscous force w . F_v of k_forces_visc.
// F_v is linear in the velocity samples:
//   w . F_v = sum_I sum_ab M_ab(I) G_ab(I),  M_ab = nu K(d_I) (w_a n_b + w_b n_a),
// with G_ab = d_b u_a the centre differences of k_forces_visc, so each sample
// that a difference reads gets M_ab times its coefficient there (1 and -1 for
// a == b, +-1/4 otherwise). Adds scale times that into (ub, ueb) through
// vel_slot (constant samples get nothing).
template <typename T, typename CS>
__global__ void k_force_visc_du(GridD g, CS cs, double w0, double w1, double w2, double scale, Vec3P<T> ub, T *ueb) {
    const double w[3] = {w0, w1, w2};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        double K, nd[3];
        if (!cs.template eval<T>(g, i, j, k, idx, K, nd)) continue;
        for (int a = 0; a < g.ndim; ++a)
            for (int b = 0; b < g.ndim; ++b) {
                const double M = scale * g.nu * K * (w[a] * nd[b] + w[b] * nd[a]);
                if (M == 0.0) continue;
                T *ua = ub.p[a];
                if (a == b) {
                    int P[3] = {i, j, k};
                    P[a] += 1;
                    add_to(vel_slot<T>(g, ua, ueb, a, P[0], P[1], P[2]), (T)M);
                    add_to(vel_slot<T>(g, ua, ueb, a, i, j, k), (T)(-M));
                } else {
                    int q1[3] = {i, j, k}, q2[3] = {i, j, k}, q3[3] = {i, j, k}, q4[3] = {i, j, k};
                    q1[b] += 1;
                    q2[a] += 1; q2[b] += 1;
                    q3[b] -= 1;
                    q4[a] += 1; q4[b] -= 1;
                    const T m = (T)(0.25 * M);
                    add_to(vel_slot<T>(g, ua, ueb, a, q1[0], q1[1], q1[2]), m);
                    add_to(vel_slot<T>(g, ua, ueb, a, q2[0], q2[1], q2[2]), m);
                    add_to(vel_slot<T>(g, ua, ueb, a, q3[0], q3[1], q3[2]), -m);
                    add_to(vel_slot<T>(g, ua, ueb, a, q4[0], q4[1], q4[2]), -m);
                }
            }
    }
}

// ------------------------------------------------ body-parameter tangents
// Tangent of the body state with respect to one motion parameter: the heave
// amplitude moves the centre by sin(omega t + phase) along the heave axis and
// its velocity by omega cos(omega t + phase); the pitch amplitude moves the
// angle by sin(omega t + phase + pi/2) and the rate by omega cos(...).
struct BodyTangent {
    double dc[3];      // centre
    double dvc[3];     // centre velocity
    double dth, dthd;  // pitch angle and rate
};

// Signed distance, normal and velocity at point x (double) and their tangents
// along dB (same formulas as body_eval, differentiated by hand).
__device__ __forceinline__ void body_tangent(const BodyState &B, const BodyTangent &dB, int ndim, const double (&x)[3],
                                             double &d, double (&n)[3], double (&V)[3], double &dd,
                                             double (&dn)[3], double (&dV)[3]) {
    double rv[3], drv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        rv[a] = a < ndim ? (x[a] - B.chi[a]) - B.clo[a] : 0.0;
        drv[a] = a < ndim ? -dB.dc[a] : 0.0;
        n[a] = dn[a] = 0.0;
        V[a] = B.vc[a];
        dV[a] = dB.dvc[a];
    }
    d = 1e30;
    dd = 0.0;
    if (B.kind == 1 || B.kind == 3) {
        if (B.kind == 3) { rv[2] = 0.0; drv[2] = 0.0; }   // cylinder: in-plane distance
        const double rr = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        d = rr - B.radius;
        if (rr > 0.0) {
            double nd = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) { n[a] = rv[a] / rr; nd += n[a] * drv[a]; }
            dd = nd;
#pragma unroll
            for (int a = 0; a < 3; ++a) dn[a] = (drv[a] - n[a] * nd) / rr;
        } else {
            n[0] = 1.0;
        }
    } else if (B.kind == 2) {
        const double ct = B.cth, st = B.sth, sa2 = B.sa * B.sa, sb2 = B.sb * B.sb;
        const double xp = ct * rv[0] + st * rv[1], yp = -st * rv[0] + ct * rv[1];
        const double dxp = ct * drv[0] + st * drv[1] + yp * dB.dth;
        const double dyp = -st * drv[0] + ct * drv[1] - xp * dB.dth;
        const double q = sqrt(xp * xp / sa2 + yp * yp / sb2);
        const double gx = xp / sa2, gy = yp / sb2;
        const double gn = sqrt(gx * gx + gy * gy);
        if (gn > 0.0) {
            const double dq = q > 0.0 ? (xp * dxp / sa2 + yp * dyp / sb2) / q : 0.0;
            const double dgx = dxp / sa2, dgy = dyp / sb2;
            const double dgn = (gx * dgx + gy * dgy) / gn;
            d = (q - 1.0) * q / gn;
            dd = ((2.0 * q - 1.0) * dq * gn - (q - 1.0) * q * dgn) / (gn * gn);
            const double nx = gx / gn, ny = gy / gn;
            const double dnx = (dgx * gn - gx * dgn) / (gn * gn), dny = (dgy * gn - gy * dgn) / (gn * gn);
            n[0] = ct * nx - st * ny;
            n[1] = st * nx + ct * ny;
            dn[0] = ct * dnx - st * dny - dB.dth * n[1];
            dn[1] = st * dnx + ct * dny + dB.dth * n[0];
        } else {
            d = -B.sb;
            n[0] = 1.0;
        }
        V[0] += -B.thd * rv[1];
        V[1] += B.thd * rv[0];
        dV[0] += -dB.dthd * rv[1] - B.thd * drv[1];
        dV[1] += dB.dthd * rv[0] + B.thd * drv[0];
    }
}

// Face fields (mu0, mu1 n, V) of component a at stored face (i,j,k) and their
// tangents along dB (double). mu0' = K, mu1' = -d K.
struct FaceTan {
    double mu0, m[3], V, dmu0, dm[3], dV;
};
__device__ __forceinline__ FaceTan face_tangent(const BodyState &B, const BodyTangent &dB, int ndim, int a, int i, int j,
                                                int k) {
    double x[3] = {i + 0.5, j + 0.5, k + 0.5};
    x[a] -= 0.5;
    double d, n[3], V[3], dd, dn[3], dV[3];
    body_tangent(B, dB, ndim, x, d, n, V, dd, dn, dV);
    FaceTan f;
    const double K = kkernel<double>(d, B.eps);
    const double m1 = kmu1<double>(d, B.eps);
    f.mu0 = kmu0<double>(d, B.eps);
    f.dmu0 = K * dd;
    if (f.mu0 < WL_MU0_MIN) { f.mu0 = 0.0; f.dmu0 = 0.0; }   // the measure's cut
    const double dm1 = -d * K * dd;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        f.m[b] = b < ndim ? m1 * n[b] : 0.0;
        f.dm[b] = b < ndim ? dm1 * n[b] + m1 * dn[b] : 0.0;
    }
    f.V = V[a];
    f.dV = dV[a];
    return f;
}

// Tangent of the blended velocity along two parameter directions, contracted
// with the blend's cotangent: acc[p] += sum_faces s gin * du/dtheta_p, with
//   du = dV + dmu0 (f - V) - mu0 dV + sum_b [dm_b (f - V)(P_b) - (f - V)(M_b)) / 2
//                                            - m_b (dV(P_b) - dV(M_b)) / 2]
// (P_b / M_b the clamped / wrapped neighbours along b). Only faces of tiles
// with non-uniform coefficients can carry a body term. Adds into out[0..1].
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_param_blend(LevelD<T> L, CVec3P<T> gin, T s, CVec3P<T> f, CVec3P<T> Vf,
                                                         BodyState B, BodyTangent dB0, BodyTangent dB1,
                                                         DevScalars *S, double *part, double *out) {
    const GridD &g = L.g;
    double acc[2] = {0.0, 0.0};
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (uni) return;
        const int J[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            if (!g.per[a] && J[a] == 0) continue;
            const double gv = (double)s * (double)gin.p[a][idx];
            if (gv == 0.0) continue;
            const FaceTan c0 = face_tangent(B, dB0, NDIM, a, i, j, k);
            if (c0.mu0 >= 1.0 && c0.dmu0 == 0.0 && c0.m[0] == 0.0 && c0.m[1] == 0.0 && c0.m[2] == 0.0) continue;
            const FaceTan c1 = face_tangent(B, dB1, NDIM, a, i, j, k);
            const double fv = (double)f.p[a][idx] - (double)Vf.p[a][idx];
            double du0 = c0.dV + c0.dmu0 * fv - c0.mu0 * c0.dV;
            double du1 = c1.dV + c1.dmu0 * fv - c1.mu0 * c1.dV;
#pragma unroll
            for (int b = 0; b < NDIM; ++b) {
                int P[3] = {i, j, k}, M[3] = {i, j, k};
                P[b] += 1;
                M[b] -= 1;
#pragma unroll
                for (int ax = 0; ax < NDIM; ++ax) {
                    const int N = g.n[ax];
                    if (g.per[ax]) { P[ax] = wrapi(P[ax], N); M[ax] = wrapi(M[ax], N); }
                    else { P[ax] = P[ax] > N - 1 ? N - 1 : P[ax]; M[ax] = M[ax] < 0 ? 0 : M[ax]; }
                }
                const long long ip = lin3(g, P[0], P[1], P[2]), im = lin3(g, M[0], M[1], M[2]);
                const double dfv = ((double)f.p[a][ip] - (double)Vf.p[a][ip]) - ((double)f.p[a][im] - (double)Vf.p[a][im]);
                const FaceTan p0 = face_tangent(B, dB0, NDIM, a, P[0], P[1], P[2]);
                const FaceTan m0 = face_tangent(B, dB0, NDIM, a, M[0], M[1], M[2]);
                const FaceTan p1 = face_tangent(B, dB1, NDIM, a, P[0], P[1], P[2]);
                const FaceTan m1 = face_tangent(B, dB1, NDIM, a, M[0], M[1], M[2]);
                du0 += 0.5 * (c0.dm[b] * dfv - c0.m[b] * (p0.dV - m0.dV));
                du1 += 0.5 * (c1.dm[b] * dfv - c1.m[b] * (p1.dV - m1.dV));
            }
            acc[0] += gv * du0;
            acc[1] += gv * du1;
        }
    });
    double red[2];
    if (grid_reduce<2, false, double>(acc, part, &S->counters[RS_MISC], red))
        if (threadIdx.x == 0 && threadIdx.y == 0) { out[0] += red[0]; out[1] += red[1]; }
}

// Tangent of the blended velocity along a body-velocity field dV at fixed
// geometry (a sampled body whose velocity depends on one parameter), contracted
// with the blend's cotangent: acc += sum_faces s gin du on the faces k_blend
// treats as body faces, with
//   du = dV - mu0 dV - sum_b mu1 n_b (dV(P_b) - dV(M_b)) / 2,
// neighbours sampled as k_blend samples f and V. Adds into out[0].
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_vtan_blend(LevelD<T> L, CVec3P<T> gin, T s, const T *mu1n0,
                                                        long long mstride, CVec3P<T> dV, DevScalars *S, double *part,
                                                        double *out) {
    const GridD &g = L.g;
    double acc[1] = {0.0};
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (uni) return;
        const int J[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            if (!g.per[a] && J[a] == 0) continue;
            const T ca = L.c[a][idx];
            bool plain = ca == L.cu;
#pragma unroll
            for (int b = 0; b < NDIM; ++b) plain = plain && mu1n0[(a * 3 + b) * mstride + idx] == T(0);
            if (plain) continue;
            const double gv = (double)s * (double)gin.p[a][idx];
            if (gv == 0.0) continue;
            const double dv = (double)dV.p[a][idx];
            double du = dv - (double)ca * dv;
#pragma unroll
            for (int b = 0; b < NDIM; ++b) {
                const T m = mu1n0[(a * 3 + b) * mstride + idx];
                if (m == T(0)) continue;
                int P[3] = {i, j, k}, M[3] = {i, j, k};
                P[b] += 1;
                M[b] -= 1;
                du -= (double)m * 0.5 *
                      ((double)face_sample<T>(g, dV.p[a], P[0], P[1], P[2]) - (double)face_sample<T>(g, dV.p[a], M[0], M[1], M[2]));
            }
            acc[0] += gv * du;
        }
    });
    double red[1];
    if (grid_reduce<1, false, double>(acc, part, &S->counters[RS_MISC], red))
        if (threadIdx.x == 0 && threadIdx.y == 0) out[0] += red[0];
}

// Coefficient part of the projection's parameter derivative: with the forward
// pressure P of the projection (pair Ph + Pl), the adjoint solution q' (pair
// qh + ql) and the cotangent lam of the projected velocity,
//   dJ/dc_a[I] = w dt (P[I] - P[I-e_a]) ((q'[I] - q'[I-e_a]) - lam_a[I]),
// contracted with dc = dmu0 on faces whose coefficient is mu0. Adds into out.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_adj_param_coef(LevelD<T> L, const T *Ph, const T *Pl, const T *qh,
                                                        const T *ql, CVec3P<T> lam, double wdt, BodyState B,
                                                        BodyTangent dB0, BodyTangent dB1, DevScalars *S, double *part,
                                                        double *out) {
    const GridD &g = L.g;
    double acc[2] = {0.0, 0.0};
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (uni) return;
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, false, i, j, k, idx, ip, im, cp, cm);
        const int I[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            if (!g.per[a] && I[a] == 0) continue;
            const FaceTan t0 = face_tangent(B, dB0, NDIM, a, i, j, k);
            const FaceTan t1 = face_tangent(B, dB1, NDIM, a, i, j, k);
            if (t0.dmu0 == 0.0 && t1.dmu0 == 0.0) continue;
            const double dP = ((double)Ph[idx] - (double)Ph[im[a]]) + ((double)Pl[idx] - (double)Pl[im[a]]);
            const double dq = ((double)qh[idx] - (double)qh[im[a]]) + ((double)ql[idx] - (double)ql[im[a]]);
            const double cb = wdt * dP * (dq - (double)lam.p[a][idx]);
            acc[0] += cb * t0.dmu0;
            acc[1] += cb * t1.dmu0;
        }
    });
    double red[2];
    if (grid_reduce<2, false, double>(acc, part, &S->counters[RS_MISC], red))
        if (threadIdx.x == 0 && threadIdx.y == 0) { out[0] += red[0]; out[1] += red[1]; }
}

// Direct parameter derivative of the weighted force w.F at fixed pressure:
// F = -sum_I (p_I - mean) n(x_I) K(d(x_I)) over active cells, so
// d(w.F) = -sum_I (p_I - mean) sum_a w_a (dn_a K + n_a K' dd). Adds into out.
template <typename T>
__global__ void k_force_dparam(GridD g, BodyState B, BodyTangent dB0, BodyTangent dB1, const T *ph, const T *pl,
                               const T *invD, double w0, double w1, double w2, DevScalars *S, double *part,
                               double *out) {
    const double pm = S->pmean;
    const double w[3] = {w0, w1, w2};
    double acc[2] = {0.0, 0.0};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        if (invD[idx] == T(0)) continue;
        int i, j, k;
        decode(g, idx, i, j, k);
        const double x[3] = {i + 0.5, j + 0.5, k + 0.5};
        const double p = ((double)ph[idx] - pm) + (double)pl[idx];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            double d, n[3], V[3], dd, dn[3], dV[3];
            body_tangent(B, q == 0 ? dB0 : dB1, g.ndim, x, d, n, V, dd, dn, dV);
            const double r = d / B.eps;
            if (!(r > -1.0 && r < 1.0)) continue;
            const double K = kkernel<double>(d, B.eps);
            const double Kp = -0.5 * 3.14159265358979323846 * sinpi(r) / (B.eps * B.eps);
            double s = 0.0;
            for (int a = 0; a < g.ndim; ++a) s += w[a] * (dn[a] * K + n[a] * Kp * dd);
            acc[q] -= p * s;
        }
    }
    double red[2];
    if (grid_reduce<2, false, double>(acc, part, &S->counters[RS_MISC], red))
        if (threadIdx.x == 0) { out[0] += red[0]; out[1] += red[1]; }
}
