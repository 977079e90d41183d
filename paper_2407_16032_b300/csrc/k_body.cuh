// k_body.cuh -- analytic body measure, BDIM blend and pressure force.
//
// Sec. 2: the momentum update is convolved with the body equation u = V
// through a kernel of half-width eps; with the signed distance d (> 0 in the
// fluid) and the normal n = grad d, the zeroth and first kernel moments are
//     mu0(d) = (1 + r + sin(pi r)/pi)/2,
//     mu1(d) = eps [1/4 - r^2/4 - (r sin(pi r) + (1 + cos(pi r))/pi)/(2 pi)],
// r = d/eps on |r| < 1 (mu0 = 0 / 1 and mu1 = 0 outside), and the blended
// velocity on face a is  u = V + mu0 (f - V) + mu1 n . grad(f - V).
// Sec. 3: bodies are a distance function plus a motion map (AutoBody); here the
// map is a rigid heave (and pitch for the 2D ellipse), evaluated per face.
#pragma once
#include "wl_common.cuh"
#include "k_poisson.cuh"

// Body state at one instant, prepared on the host in double precision.
// The centre is split into an integer part and a remainder so that face
// offsets x - c stay accurate in single precision.
struct BodyState {
    int kind;          // 0 none, 1 sphere/circle, 2 ellipse (2D), 3 cylinder along z (3D)
    double chi[3];     // integer part of the centre
    double clo[3];     // centre - chi
    double radius;
    double sa, sb;     // ellipse semi-axes
    double cth, sth;   // cos / sin of the pitch angle
    double vc[3];      // centre velocity
    double thd;        // pitch rate
    double eps;
};

__device__ __forceinline__ float sinpi_t(float x) { return sinpif(x); }
__device__ __forceinline__ double sinpi_t(double x) { return sinpi(x); }
__device__ __forceinline__ float cospi_t(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_t(double x) { return cospi(x); }

template <typename T>
__device__ __forceinline__ T kmu0(T d, T eps) {
    const T r = d / eps;
    if (r <= T(-1)) return T(0);
    if (r >= T(1)) return T(1);
    return T(0.5) * (T(1) + r + sinpi_t(r) * T(0.31830988618379067154));
}
template <typename T>
__device__ __forceinline__ T kmu1(T d, T eps) {
    const T r = d / eps;
    if (r <= T(-1) || r >= T(1)) return T(0);
    const T ip = T(0.31830988618379067154);
    return eps * (T(0.25) - T(0.25) * r * r - (r * sinpi_t(r) + (T(1) + cospi_t(r)) * ip) * (T(0.5) * ip));
}
// Smallest zeroth moment kept on a face: below it the face counts as solid
// (mu0 = 0). A cell whose faces sum to a tiny nonzero coefficient has a
// pressure fixed only by its right-hand side's rounding divided by that sum,
// yet counts in the mean over active rows; the cut trims the outermost few
// percent of the kernel's reach (mu0 ~ pi^2 (1 + r)^3 / 12 near r = -1).
#define WL_MU0_MIN 1e-5
__device__ __forceinline__ double mu0_kept(double m) { return m < WL_MU0_MIN ? 0.0 : m; }

template <typename T>
__device__ __forceinline__ T kkernel(T d, T eps) {
    const T r = d / eps;
    if (r <= T(-1) || r >= T(1)) return T(0);
    return (T(1) + cospi_t(r)) / (T(2) * eps);
}

// Signed distance, normal and velocity of the body at point p = (cell index
// + offsets) given as exact small values px (offsets from the integer centre
// are formed before the remainder is removed).
template <typename T>
__device__ __forceinline__ void body_eval(const BodyState &B, int ndim, const T (&px)[3], T &d, T (&nrm)[3], T (&V)[3]) {
    T rv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        rv[a] = a < ndim ? (px[a] - (T)B.chi[a]) - (T)B.clo[a] : T(0);
        nrm[a] = T(0);
        V[a] = (T)B.vc[a];
    }
    if (B.kind == 1 || B.kind == 3) {
        if (B.kind == 3) rv[2] = T(0);   // cylinder: distance in the x-y plane
        T r2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
        T rr = sqrt(r2);
        d = rr - (T)B.radius;
        if (rr > T(0)) {
            const T inv = T(1) / rr;
#pragma unroll
            for (int a = 0; a < 3; ++a) nrm[a] = rv[a] * inv;
        } else {
            nrm[0] = T(1);
        }
    } else if (B.kind == 2) {
        const T ct = (T)B.cth, st = (T)B.sth, sa = (T)B.sa, sb = (T)B.sb;
        const T xp = ct * rv[0] + st * rv[1], yp = -st * rv[0] + ct * rv[1];
        const T q = sqrt((xp / sa) * (xp / sa) + (yp / sb) * (yp / sb));
        const T gx = xp / (sa * sa), gy = yp / (sb * sb);
        const T gn = sqrt(gx * gx + gy * gy);
        if (gn > T(0)) {
            d = (q - T(1)) * q / gn;
            const T nx = gx / gn, ny = gy / gn;
            nrm[0] = ct * nx - st * ny;
            nrm[1] = st * nx + ct * ny;
        } else {
            d = -sb;
            nrm[0] = T(1);
        }
        V[0] += -(T)B.thd * rv[1];
        V[1] += (T)B.thd * rv[0];
    } else {
        d = T(1e30);
    }
}

// Measure every stored face: c_a = mu0 (0 on lower faces of non-periodic axes),
// mu1n[a*3+b] = mu1 n_b, V[a] = body velocity component a.
// On the cells of box b only, one (tile, plane) item per block.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_measure(LevelD<T> L, BodyState B, Vec3P<T> c, T *mu1n0, long long mstride,
                                                 Vec3P<T> V, bool full, CellBox box) {
    const T eps = (T)B.eps;
    const GridD &g = L.g;
    for_box_planes<NDIM>(g, box, [&](int i, int j, int k, long long idx) {
        const int I[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            T px[3] = {T(i) + T(0.5), T(j) + T(0.5), T(k) + T(0.5)};
            px[a] -= T(0.5);
            T d, nrm[3], v[3];
            body_eval<T>(B, NDIM, px, d, nrm, v);
            T m0 = (T)mu0_kept((double)kmu0<T>(d, eps)), m1 = kmu1<T>(d, eps);
            if (sizeof(T) < sizeof(double) && d > -eps - T(0.5) && d < eps + T(0.5)) {
                // inside the kernel band: distance, normal and moments in double
                // (a thin shell of faces), rounded once to T
                double pd[3] = {i + 0.5, j + 0.5, k + 0.5}, dd, nd[3], vd[3];
                pd[a] -= 0.5;
                body_eval<double>(B, NDIM, pd, dd, nd, vd);
                m0 = (T)mu0_kept(kmu0<double>(dd, B.eps));
                m1 = (T)kmu1<double>(dd, B.eps);
#pragma unroll
                for (int b = 0; b < 3; ++b) { nrm[b] = (T)nd[b]; v[b] = (T)vd[b]; }
            }
            c.p[a][idx] = (!g.per[a] && I[a] == 0) ? T(0) : m0;
            if (full) {
#pragma unroll
                for (int b = 0; b < NDIM; ++b) mu1n0[(a * 3 + b) * mstride + idx] = m1 * nrm[b];
                V.p[a][idx] = v[a];
            }
        }
    });
}

// Moments of a body given by samples (Sec. 3 states a body as a distance
// function and a map; here the caller evaluates them): on entry c.p[a] holds
// the signed distance at face a and mu1n slot a*NDIM+b the normal component b
// there; on return c.p[a] = mu0(d) (cut below WL_MU0_MIN; 0 on lower faces of
// non-periodic axes) and
// slot a*3+b = mu1(d) n_b (0 for b >= NDIM), both formed in double from the
// stored samples and rounded once to T. Every cell is read before it is
// written, by the thread that owns it.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_measure_sampled(GridD g, Vec3P<T> c, T *mu1n0, long long mstride, double eps) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        const int I[3] = {i, j, k};
        double d[NDIM], n[NDIM][NDIM];
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            d[a] = (double)c.p[a][idx];
#pragma unroll
            for (int b = 0; b < NDIM; ++b) n[a][b] = (double)mu1n0[(a * NDIM + b) * mstride + idx];
        }
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const double m1 = kmu1<double>(d[a], eps);
            c.p[a][idx] = (!g.per[a] && I[a] == 0) ? T(0) : (T)mu0_kept(kmu0<double>(d[a], eps));
#pragma unroll
            for (int b = 0; b < 3; ++b) mu1n0[(a * 3 + b) * mstride + idx] = b < NDIM ? (T)(m1 * n[a][b]) : T(0);
        }
    }
}

// Kernel weight K_eps(d) and unit normal at the centre of cell (i, j, k):
// false where K is zero. Analytic bodies evaluate the distance in T first
// and only inside the band (with half a cell of margin) again in double;
// sampled bodies read the caller's centre samples.
struct CentreAnalytic {
    BodyState B;
    template <typename T>
    __device__ __forceinline__ bool eval(const GridD &g, int i, int j, int k, long long, double &K, double (&n)[3]) const {
        const T eps = (T)B.eps;
        T px[3] = {T(i) + T(0.5), T(j) + T(0.5), T(k) + T(0.5)};
        T d, nrm[3], v[3];
        body_eval<T>(B, g.ndim, px, d, nrm, v);
        if (!(d > -eps - T(0.5) && d < eps + T(0.5))) return false;
        double pd[3] = {i + 0.5, j + 0.5, k + 0.5}, dd, vd[3];
        body_eval<double>(B, g.ndim, pd, dd, n, vd);
        K = kkernel<double>(dd, B.eps);
        return K != 0.0;
    }
};
template <typename TS> struct CentreSampled {
    const TS *d;       // signed distance at the cell centres
    const TS *n[3];    // unit normal components at the cell centres
    double eps;
    template <typename T>
    __device__ __forceinline__ bool eval(const GridD &g, int, int, int, long long idx, double &K, double (&nv)[3]) const {
        K = kkernel<double>((double)d[idx], eps);
        if (K == 0.0) return false;
#pragma unroll
        for (int a = 0; a < 3; ++a) nv[a] = a < g.ndim ? (double)n[a][idx] : 0.0;
        return true;
    }
};

// BDIM blend of the stage value f (Sec. 2): u = V + mu0 (f - V) + mu1 n.grad(f - V);
// corrector stage averages with u*: u = (u* + blend)/2; lower boundary faces of
// non-periodic axes take U_a. Tiles flagged uniform (no body face in the tile
// or its halo) have mu0 = 1, mu1 = 0 and skip the body arrays, and so do fluid
// faces outside the kernel band (mu0 = 1, mu1 = 0): there u = f.
template <typename T, int NDIM, bool CORR>
__global__ void __launch_bounds__(256) k_blend(LevelD<T> L, CVec3P<T> f, const T *mu1n0, long long mstride,
                                               CVec3P<T> V, CVec3P<T> ustar, Vec3P<T> out) {
    const GridD &g = L.g;
    for_cells<NDIM>(g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        const int I[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const T fa = f.p[a][idx];
            T val;
            bool plain = uni || L.c[a][idx] == L.cu;
            if (!uni)
#pragma unroll
                for (int b = 0; b < NDIM; ++b) plain = plain && mu1n0[(a * 3 + b) * mstride + idx] == T(0);
            if (plain) {
                // no body face within a cell, or a fluid face outside the
                // kernel band: the blend is f itself (no body velocity read)
                val = fa;
            } else {
                const T Va = V.p[a][idx];
                T grad = T(0);
#pragma unroll
                for (int b = 0; b < NDIM; ++b) {
                    const T m = mu1n0[(a * 3 + b) * mstride + idx];
                    if (m != T(0)) {
                        int P[3] = {i, j, k}, M[3] = {i, j, k};
                        P[b] += 1;
                        M[b] -= 1;
                        const T up = face_sample<T>(g, f.p[a], P[0], P[1], P[2]) - face_sample<T>(g, V.p[a], P[0], P[1], P[2]);
                        const T dn = face_sample<T>(g, f.p[a], M[0], M[1], M[2]) - face_sample<T>(g, V.p[a], M[0], M[1], M[2]);
                        grad += m * T(0.5) * (up - dn);
                    }
                }
                val = Va + L.c[a][idx] * (fa - Va) + grad;
            }
            if (CORR) val = T(0.5) * (ustar.p[a][idx] + val);
            if (!g.per[a] && I[a] == 0) val = (T)g.U[a];
            out.p[a][idx] = val;
        }
    });
}

// The blend on the tiles flagged non-uniform only (the tiles within a cell of
// a body face; elsewhere the blend is the identity and the flux kernel wrote
// the stage's final value, FM_PRED_M / FM_CORR_M): the blend of k_blend into
// `out` at those tiles' cells; fluid faces outside the kernel band (c = cu,
// mu1 = 0) take f itself and read no body velocity. The blend's neighbour
// samples of f lie in flagged tiles too (mu1 != 0 only within the kernel band).
template <typename T, int NDIM, bool CORR>
__global__ void __launch_bounds__(256) k_blend_band(LevelD<T> L, CVec3P<T> f, const T *mu1n0, long long mstride,
                                                    CVec3P<T> V, CVec3P<T> ustar, Vec3P<T> out, const int *tlist,
                                                    const unsigned *tcount) {
    const GridD &g = L.g;
    // work items: (listed tile, plane of the tile)
    const int nb = (int)*tcount * MT<NDIM>::TZ;
    for (int q = blockIdx.x; q < nb; q += gridDim.x) {
        const int t = tlist[q / MT<NDIM>::TZ];
        const int bx = t % L.tl.ntx, rr = t / L.tl.ntx;
        const int by = rr % L.tl.nty, bz = rr / L.tl.nty;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y;
        if (i >= g.n[0] || j >= g.n[1]) continue;
        {
            const int k = bz * MT<NDIM>::TZ + q % MT<NDIM>::TZ;
            if (k >= g.n[2]) continue;
            const long long idx = (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
            const int I[3] = {i, j, k};
#pragma unroll
            for (int a = 0; a < NDIM; ++a) {
                const T fa = f.p[a][idx];
                const T ca = L.c[a][idx];
                bool plain = ca == L.cu;
#pragma unroll
                for (int b = 0; b < NDIM; ++b) plain = plain && mu1n0[(a * 3 + b) * mstride + idx] == T(0);
                if (plain) {
                    // a fluid face outside the kernel band: the blend is f itself
                    T val = fa;
                    if (CORR) val = T(0.5) * (ustar.p[a][idx] + val);
                    if (!g.per[a] && I[a] == 0) val = (T)g.U[a];
                    out.p[a][idx] = val;
                    continue;
                }
                const T Va = V.p[a][idx];
                T grad = T(0);
#pragma unroll
                for (int b = 0; b < NDIM; ++b) {
                    const T m = mu1n0[(a * 3 + b) * mstride + idx];
                    if (m != T(0)) {
                        int Pp[3] = {i, j, k}, M[3] = {i, j, k};
                        Pp[b] += 1;
                        M[b] -= 1;
                        const T up = face_sample<T>(g, f.p[a], Pp[0], Pp[1], Pp[2]) - face_sample<T>(g, V.p[a], Pp[0], Pp[1], Pp[2]);
                        const T dn = face_sample<T>(g, f.p[a], M[0], M[1], M[2]) - face_sample<T>(g, V.p[a], M[0], M[1], M[2]);
                        grad += m * T(0.5) * (up - dn);
                    }
                }
                T val = Va + ca * (fa - Va) + grad;
                if (CORR) val = T(0.5) * (ustar.p[a][idx] + val);
                if (!g.per[a] && I[a] == 0) val = (T)g.U[a];
                out.p[a][idx] = val;
            }
        }
    }
}

// Copy the cells of the tiles flagged non-uniform (the list) from src to dst.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_band_copy(LevelD<T> L, CVec3P<T> src, Vec3P<T> dst, const int *tlist,
                                                   const unsigned *tcount) {
    const GridD &g = L.g;
    // work items: (listed tile, plane of the tile)
    const int nb = (int)*tcount * MT<NDIM>::TZ;
    for (int q = blockIdx.x; q < nb; q += gridDim.x) {
        const int t = tlist[q / MT<NDIM>::TZ];
        const int bx = t % L.tl.ntx, rr = t / L.tl.ntx;
        const int by = rr % L.tl.nty, bz = rr / L.tl.nty;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y;
        if (i >= g.n[0] || j >= g.n[1]) continue;
        {
            const int k = bz * MT<NDIM>::TZ + q % MT<NDIM>::TZ;
            if (k >= g.n[2]) continue;
            const long long idx = (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
#pragma unroll
            for (int a = 0; a < NDIM; ++a) dst.p[a][idx] = src.p[a][idx];
        }
    }
}

// The tiles flagged non-uniform, appended to tlist (in no particular order;
// each tile's blend is independent of the others'); *tcount starts at 0.
static __global__ void __launch_bounds__(256) k_tile_list(const unsigned char *tflag, int nt, int *tlist, unsigned *tcount) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x)
        if (!tflag[t]) tlist[atomicAdd(tcount, 1u)] = t;
}

// Pressure force F = -sum_I (p_I - pmean) n(x_I) K_eps(d(x_I)) over active cells.
template <typename T, typename CS>
__global__ void k_forces(GridD g, CS cs, const T *ph, const T *pl, const T *invD, DevScalars *S, double *part) {
    const T pm = (T)S->pmean;
    T acc[3] = {T(0), T(0), T(0)};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        if (invD[idx] == T(0)) continue;
        double Kd, nd[3];
        if (!cs.template eval<T>(g, i, j, k, idx, Kd, nd)) continue;
        const T K = (T)Kd;
        if (K == T(0)) continue;
        T nrm[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) nrm[a] = (T)nd[a];
        const T p = (ph[idx] - pm) + pl[idx];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] -= p * K * nrm[a];
    }
    double out[3];
    if (grid_reduce<3, false, T>(acc, part, &S->counters[RS_FORCE], out)) {
        if (threadIdx.x == 0) { S->red[0] = out[0]; S->red[1] = out[1]; S->red[2] = out[2]; }
    }
}

// Viscous force F_a = nu sum_I K_eps(d(x_I)) sum_b S_ab(x_I) n_b(x_I) over cell
// centres: the viscous part of the stress traction on the body (n = grad d
// points into the fluid, as in the pressure part), S = grad u + grad u^T at the
// centre from the face samples,
//   d_a u_a = u_a[I+e_a] - u_a[I],
//   d_b u_a = ((u_a[I+e_b] + u_a[I+e_a+e_b]) - (u_a[I-e_b] + u_a[I+e_a-e_b])) / 4  (b != a),
// samples beyond the stored range by the boundary rule of vel_sample.
template <typename T, typename CS>
__global__ void k_forces_visc(GridD g, CS cs, CVec3P<T> u, const T *ue, DevScalars *S, double *part) {
    T acc[3] = {T(0), T(0), T(0)};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        decode(g, idx, i, j, k);
        double K, nd[3];
        if (!cs.template eval<T>(g, i, j, k, idx, K, nd)) continue;
        T G[3][3];   // G[a][b] = d_b u_a
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                G[a][b] = T(0);
                if (a >= g.ndim || b >= g.ndim) continue;
                const T *ua = u.p[a];
                if (a == b) {
                    int P[3] = {i, j, k};
                    P[a] += 1;
                    G[a][b] = vel_sample<T>(g, ua, ue, a, P[0], P[1], P[2]) - vel_sample<T>(g, ua, ue, a, i, j, k);
                } else {
                    int q1[3] = {i, j, k}, q2[3] = {i, j, k}, q3[3] = {i, j, k}, q4[3] = {i, j, k};
                    q1[b] += 1;              // I + e_b
                    q2[a] += 1; q2[b] += 1;  // I + e_a + e_b
                    q3[b] -= 1;              // I - e_b
                    q4[a] += 1; q4[b] -= 1;  // I + e_a - e_b
                    const T up = vel_sample<T>(g, ua, ue, a, q1[0], q1[1], q1[2]) +
                                 vel_sample<T>(g, ua, ue, a, q2[0], q2[1], q2[2]);
                    const T dn = vel_sample<T>(g, ua, ue, a, q3[0], q3[1], q3[2]) +
                                 vel_sample<T>(g, ua, ue, a, q4[0], q4[1], q4[2]);
                    G[a][b] = T(0.25) * (up - dn);
                }
            }
        const T nuK = (T)(g.nu * K);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= g.ndim) continue;
            T tr = T(0);
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (b < g.ndim) tr += (G[a][b] + G[b][a]) * (T)nd[b];
            acc[a] += nuK * tr;
        }
    }
    double out[3];
    if (grid_reduce<3, false, T>(acc, part, &S->counters[RS_FORCE], out)) {
        if (threadIdx.x == 0) { S->red[0] = out[0]; S->red[1] = out[1]; S->red[2] = out[2]; }
    }
}
