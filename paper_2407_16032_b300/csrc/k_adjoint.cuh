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

// Pressure derivative of the force on the body, component `axis`:
// F = -sum_I (p_I - mean) n(x_I) K_eps(d(x_I)) over active cells, so
// dF/dp_I = -n_axis K on active cells of the kernel band (the mean's share is
// removed by the adjoint solve, whose right-hand side is made mean-free).
template <typename T>
__global__ void k_force_dp(GridD g, BodyState B, const T *invD, int axis, double scale, double *out) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        double v = 0.0;
        if (invD[idx] != T(0)) {
            double pd[3] = {i + 0.5, j + 0.5, k + 0.5}, dd, nd[3], vd[3];
            body_eval<double>(B, g.ndim, pd, dd, nd, vd);
            v = -scale * nd[axis] * kkernel<double>(dd, B.eps);
        }
        out[idx] = v;
    }
}
