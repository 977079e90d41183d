// k_misc.cuh -- convective exit, CFL time step and diagnostics kernels.
#pragma once
#include "wl_common.cuh"
#include "k_poisson.cuh"

// Convective outlet on the upper x face (Sec. 4: convective outflow boundary).
// The exit face value follows du/dt + U du/dx = 0 with a first-order upwind
// difference against the last interior u_x face, advanced by the same Heun
// stages as the interior:
//   predictor  ue = ue0 + dt G(ueG, uG)        corrector  ue = (ue* + ue0 + dt G(ueG, uG))/2
//   G = -U_x (ueG - uG_x[n0-1]);
// then a uniform correction makes the net boundary volume flux zero: with all
// other boundary normals at U, that is ue += U_x - mean(ue). One block.
template <typename T, bool CORR>
__global__ void k_exit(GridD g, const T *ue0, const T *uGx, const T *ueG, const T *uestar, T dt, T *ue) {
    const int np = g.n[1] * (g.ndim == 3 ? g.n[2] : 1);
    const int n0 = g.n[0];
    const T Ub = (T)g.U[0];
    __shared__ double sh[32];
    T acc[1] = {T(0)};
    double out[1];
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const T last = uGx[(long long)(n0 - 1) + (long long)n0 * p];
        const T G = -Ub * (ueG[p] - last);
        T v = ue0[p] + dt * G;
        if (CORR) v = T(0.5) * (uestar[p] + v);
        ue[p] = v;
        acc[0] += v;
    }
    block_reduce<1, false, T>(acc, out, sh);
    if (threadIdx.x == 0) sh[0] = out[0];
    __syncthreads();
    const T corr = (T)((double)g.U[0] - sh[0] / (double)np);
    for (int p = threadIdx.x; p < np; p += blockDim.x) ue[p] += corr;
}

// Lower boundary faces of the non-periodic axes carry the free stream U_a.
template <typename T>
__global__ void k_bc_lower(GridD g, Vec3P<T> u) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int I[3];
        decode(g, idx, I[0], I[1], I[2]);
        for (int a = 0; a < g.ndim; ++a)
            if (!g.per[a] && I[a] == 0) u.p[a][idx] = (T)g.U[a];
    }
}

// Fill a plane with a constant.
// y += alpha x over n elements.
template <typename T>
__global__ void k_axpy(long long n, T alpha, const T *x, T *y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += alpha * x[i];
}

template <typename T>
__global__ void k_fill(long long n, T v, T *x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = v;
}

// CFL time step (Sec. 2: the time step adapts to keep the CFL number stable):
// dt = min(dt_max, cfl / (max_I sum_a [max(0,u_a[I+e_a]) - min(0,u_a[I])] + 5 nu)).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_cfl(LevelD<T> L, CVec3P<T> u, const T *ue, double cfl, double dt_max,
                                             DevScalars *S, double *part) {
    const GridD &g = L.g;
    T acc[1] = {T(0)};
    for_cells<NDIM>(g, L.tl, nullptr, [&](int i, int j, int k, long long idx, bool) {
        const int I[3] = {i, j, k};
        const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
        T s = T(0);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            T up;
            if (I[a] + 1 < g.n[a]) up = u.p[a][idx + st[a]];
            else if (g.per[a]) up = u.p[a][idx - (long long)(g.n[a] - 1) * st[a]];
            else up = (a == 0 && g.exit_x) ? ue[j + (long long)g.n[1] * k] : (T)g.U[a];
            const T lo = u.p[a][idx];
            s += (up > T(0) ? up : T(0)) - (lo < T(0) ? lo : T(0));
        }
        acc[0] = s > acc[0] ? s : acc[0];
    });
    double out[1];
    if (grid_reduce<1, true, T>(acc, part, &S->counters[RS_CFL], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            S->maxflux = out[0];
            const double dt = cfl / (out[0] + 5.0 * g.nu);
            S->dt_next = dt < dt_max ? dt : dt_max;
        }
}

// Kinetic energy (cell-centred |u|^2/2), squared vorticity on cell edges, and
// max |div u| over active rows; results into S->red[0..2] (means / max).
template <typename T>
__global__ void k_diag(GridD g, CVec3P<T> u, const T *ue, const T *invD, DevScalars *S, double *part) {
    T acc[2] = {T(0), T(0)};
    T mx[1] = {T(0)};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        T div = T(0);
        for (int a = 0; a < g.ndim; ++a) {
            int P[3] = {i, j, k};
            P[a] += 1;
            const T up = vel_sample<T>(g, u.p[a], ue, a, P[0], P[1], P[2]);
            const T lo = u.p[a][idx];
            const T uc = T(0.5) * (up + lo);
            acc[0] += T(0.5) * uc * uc;
            div += up - lo;
        }
        for (int e = 0; e < 3; ++e) {
            if (g.ndim == 2 && e != 2) continue;
            const int a = (e + 1) % 3, b = (e + 2) % 3;
            int Ma[3] = {i, j, k}, Mb[3] = {i, j, k};
            Ma[a] -= 1;
            Mb[b] -= 1;
            const T om = (u.p[b][idx] - vel_sample<T>(g, u.p[b], ue, b, Ma[0], Ma[1], Ma[2])) -
                         (u.p[a][idx] - vel_sample<T>(g, u.p[a], ue, a, Mb[0], Mb[1], Mb[2]));
            acc[1] += om * om;
        }
        if (invD[idx] != T(0)) {
            const T ad = div < T(0) ? -div : div;
            mx[0] = ad > mx[0] ? ad : mx[0];
        }
    }
    double out[2], om[1];
    if (grid_reduce<2, false, T>(acc, part, &S->counters[RS_DIAG], out))
        if (threadIdx.x == 0) { S->red[0] = out[0] / (double)g.nc; S->red[1] = out[1] / (double)g.nc; }
    if (grid_reduce<1, true, T>(mx, part + 2 * WL_MAXPART, &S->counters[RS_MISC], om))
        if (threadIdx.x == 0) S->red[2] = om[0];
}
