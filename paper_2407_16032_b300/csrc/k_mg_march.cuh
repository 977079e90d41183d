// k_mg_march.cuh -- column-marching 7-point stencils of the V-cycle.
//
// The operator is the variable-coefficient Poisson operator of the projection
// (Sec. 2; Sec. 3: u[I,i] -= c[I,i](p[I]-p[I-d(i)]) is its gradient half):
//   (A p)[I] = sum_a c_a[I+e_a](p[I+e_a]-p[I]) - c_a[I](p[I]-p[I-e_a]).
// Each thread of a 32x8 block owns one (x, y) column of a 32 x 8 x TZ tile and
// walks it along z: the z neighbours rotate through registers (one new load per
// plane), the x and y neighbours are read through L1 at offsets formed once per
// column (wrapped on periodic axes, clamped elsewhere where the coefficient is
// 0), and there is no shared-memory staging or barrier in the march.
#pragma once
#include "k_poisson.cuh"

// Index along an axis of N cells: periodic axes wrap (any distance), others clamp.
__device__ __forceinline__ int edge_idx(int v, int N, bool per) {
    if (v >= 0 && v < N) return v;
    if (per) {
        const int r = v % N;
        return r < 0 ? r + N : r;
    }
    return v < 0 ? 0 : N - 1;
}

// Per-column set-up: cell (i, j) of the plane and the in-plane offsets of its
// x and y neighbours.
struct Col {
    int i, j, oxm, oxp, oym, oyp;
    bool in;
};

__device__ __forceinline__ Col column(const GridD &g, int x0, int y0) {
    Col c;
    c.i = x0 + threadIdx.x;
    c.j = y0 + threadIdx.y;
    c.in = c.i < g.n[0] && c.j < g.n[1];
    const int i = c.in ? c.i : 0, j = c.in ? c.j : 0;
    const bool px = g.per[0] != 0, py = g.per[1] != 0;
    c.oxm = edge_idx(i - 1, g.n[0], px) - i;
    c.oxp = edge_idx(i + 1, g.n[0], px) - i;
    c.oym = (edge_idx(j - 1, g.n[1], py) - j) * g.n[0];
    c.oyp = (edge_idx(j + 1, g.n[1], py) - j) * g.n[0];
    return c;
}

// Face coefficients of cell (i,j,k) = idx: uniform tiles from the position,
// others loaded (32-bit indices: the grid has fewer than 2^31 cells).
template <typename T, int NDIM>
__device__ __forceinline__ void coefs(const LevelD<T> &L, bool uni, int i, int j, int k, int idx, T (&cp)[3],
                                      T (&cm)[3]) {
    const int I[3] = {i, j, k};
    const int st[3] = {1, L.g.n[0], L.g.n[0] * L.g.n[1]};
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const int N = L.g.n[a];
        const bool per = L.g.per[a] != 0, top = I[a] == N - 1, bot = I[a] == 0;
        if (uni) {
            cp[a] = (top && !per) ? T(0) : L.cu;
            cm[a] = (bot && !per) ? T(0) : L.cu;
        } else {
            cp[a] = top ? (per ? L.c[a][idx - (N - 1) * st[a]] : T(0)) : L.c[a][idx + st[a]];
            cm[a] = L.c[a][idx];
        }
    }
}


// Search direction and operator in one pass (a PCG iteration's first half):
//   d = D^-1 s + beta d_old   (d = D^-1 s on the first iteration),
//   q = A d,   alpha = rho / <d, q>.
// d_old and d are different buffers (dold, dnew): a tile's ring reads d_old of
// the neighbouring tiles while they write their d. Each thread owns one
// (x, y) column of a 32 x 8 x TZ tile and issues all its column's loads (s and
// d_old over TZ + 2 planes) before forming d into a shared (TZ + 2) x 10 x 34
// tile; the in-plane ring is formed by warps 0 and 7 (rows below / above the
// tile) and 16 lanes of warp 1 (columns left / right), each loading its ring
// cell over the TZ planes at once. After one barrier the operator is applied
// from shared memory. Uniform tiles form 1/D and the coefficients from the
// position.
template <typename T, int NDIM>
__device__ __forceinline__ void pcg_dq_run(const LevelD<T> &L, const T *__restrict__ dold, T *__restrict__ dnew,
                                           DevScalars *S, double *part, int lev, const bool FIRST) {
    constexpr int TZ = MT<NDIM>::TZ;
    constexpr int PZ = NDIM == 3 ? TZ + 2 : 1;   // planes held (with the z ring)
    constexpr int Z0 = NDIM == 3 ? 1 : 0;        // smem plane of the tile's first plane
    // two shared tiles, used by alternate tiles of the block: a tile's writes
    // reuse a buffer last read two tiles ago, before the previous tile's
    // barrier, so one barrier per tile suffices
    __shared__ T sdb[2][PZ][10][34];
    int tpar = 0;
    __shared__ T idtab[8];
    const GridD &g = L.g;
    const T beta = FIRST ? T(0) : (T)S->beta[lev];
    const T *__restrict__ s = L.s;
    const T *__restrict__ iD = L.invD;
    T *__restrict__ q = L.q;
    const int n0 = g.n[0], n1 = g.n[1], plane = g.n[0] * g.n[1];
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // 1/D of a uniform-tile cell: -1 / (faces * cu), faces = 2n minus its
    // non-periodic domain faces
    if (tx < 8 && ty == 0) idtab[tx] = tx > 0 ? T(-1) / (T(tx) * L.cu) : T(0);
    __syncthreads();
    auto idu = [&](int ii, int jj, int kk) -> T {
        const int I[3] = {ii, jj, kk};
        int nf = 2 * NDIM;
#pragma unroll
        for (int a = 0; a < NDIM; ++a)
            if (!g.per[a]) nf -= (I[a] == 0) + (I[a] == g.n[a] - 1);
        return idtab[nf];
    };
    T acc[1] = {T(0)};
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int nx = min(32, n0 - x0), ny = min(8, n1 - y0);
        const int zb = NDIM == 3 ? z0 : 0, nz = NDIM == 3 ? min(TZ, g.n[2] - z0) : 1;
        const int i = x0 + tx, j = y0 + ty;
        const bool in = tx < nx && ty < ny;
        // uniform tiles away from every non-periodic domain face take one 1/D
        const bool plain = uni && (px || (x0 > 0 && x0 + nx < n0)) && (py || (y0 > 0 && y0 + ny < n1)) &&
                           (NDIM == 2 || pz || (zb > 0 && zb + nz < g.n[2]));
        const T idc = idtab[2 * NDIM];
        auto dform = [&](int id, int ii, int jj, int kk, T sv, T dv) -> T {
            const T iv = !uni ? iD[id] : (plain ? idc : idu(ii, jj, kk));
            return FIRST ? iv * sv : iv * sv + beta * dv;
        };
        // ring work. 2D (one plane): warps 0 and 7 take the rows below and
        // above the tile, lanes 0..15 of warp 1 its left and right columns.
        // 3D: spread over all warps: warp w takes two planes (2 (w mod 4) and
        // the next) of the row below (w < 4) or above (w >= 4), and lanes
        // 0..15 of warp w the left / right column cells of plane w.
        int rrow = -1, rrj = 0, rsy = 0, rp0 = 0;       // row cell (x = i), planes rp0, rp0 + 1
        int rcol = -1, rci = 0, rcj = 0, rcy = 0, rcx = 0;  // column cell, plane ty
        if (NDIM == 3) {
            if (tx < nx) {
                rrow = ty < 4 ? 0 : 1;
                rrj = rrow == 0 ? edge_idx(y0 - 1, n1, py) : edge_idx(y0 + ny, n1, py);
                rsy = rrow == 0 ? 0 : ny + 1;
                rp0 = 2 * (ty & 3);
            }
            if (tx < 16 && (tx & 7) < ny && ty < nz) {
                rcol = tx < 8 ? 0 : 1;
                rci = rcol == 0 ? edge_idx(x0 - 1, n0, px) : edge_idx(x0 + nx, n0, px);
                rcj = y0 + (tx & 7);
                rcy = (tx & 7) + 1;
                rcx = rcol == 0 ? 0 : nx + 1;
            }
        } else {
            if (ty == 0 && tx < nx) { rrow = 0; rrj = edge_idx(y0 - 1, n1, py); rsy = 0; }
            else if (ty == 7 && tx < nx) { rrow = 1; rrj = edge_idx(y0 + ny, n1, py); rsy = ny + 1; }
            else if (ty == 1 && tx < 16 && (tx & 7) < ny) {
                rcol = tx < 8 ? 0 : 1;
                rci = rcol == 0 ? edge_idx(x0 - 1, n0, px) : edge_idx(x0 + nx, n0, px);
                rcj = y0 + (tx & 7);
                rcy = (tx & 7) + 1;
                rcx = rcol == 0 ? 0 : nx + 1;
            }
        }
        const int NRP = NDIM == 3 ? 2 : 1;              // row planes per thread
        T(*sd)[10][34] = sdb[tpar];
        tpar ^= 1;
        int kz[PZ];
#pragma unroll
        for (int t = 0; t < PZ; ++t) kz[t] = NDIM == 3 ? edge_idx(zb - 1 + t, g.n[2], pz) : 0;
        T sv[PZ], dv[PZ], rs[2], rd[2], cs = T(0), cd = T(0);
        // all loads of the column and of the ring cells first
        if (in) {
#pragma unroll
            for (int t = 0; t < PZ; ++t)
                if (t < nz + 2 * Z0) {
                    const int id = i + n0 * j + plane * kz[t];
                    sv[t] = s[id];
                    dv[t] = FIRST ? T(0) : dold[id];
                }
        }
        if (rrow >= 0) {
#pragma unroll
            for (int h = 0; h < NRP; ++h)
                if (rp0 + h < nz) {
                    const int kk = NDIM == 3 ? edge_idx(zb + rp0 + h, g.n[2], pz) : 0;   // (no run-time index into kz)
                    const int id = i + n0 * rrj + plane * kk;
                    rs[h] = s[id];
                    rd[h] = FIRST ? T(0) : dold[id];
                }
        }
        const int cz = NDIM == 3 ? ty : 0;
        if (rcol >= 0) {
            const int kk = NDIM == 3 ? edge_idx(zb + cz, g.n[2], pz) : 0;
            const int id = rci + n0 * rcj + plane * kk;
            cs = s[id];
            cd = FIRST ? T(0) : dold[id];
        }
        if (in) {
#pragma unroll
            for (int t = 0; t < PZ; ++t)
                if (t < nz + 2 * Z0)
                    sd[t][ty + 1][tx + 1] = dform(i + n0 * j + plane * kz[t], i, j, kz[t], sv[t], dv[t]);
        }
        if (rrow >= 0) {
#pragma unroll
            for (int h = 0; h < NRP; ++h)
                if (rp0 + h < nz) {
                    const int kk = NDIM == 3 ? edge_idx(zb + rp0 + h, g.n[2], pz) : 0;
                    sd[rp0 + h + Z0][rsy][tx + 1] = dform(i + n0 * rrj + plane * kk, i, rrj, kk, rs[h], rd[h]);
                }
        }
        if (rcol >= 0) {
            const int kk = NDIM == 3 ? edge_idx(zb + cz, g.n[2], pz) : 0;
            sd[cz + Z0][rcy][rcx] = dform(rci + n0 * rcj + plane * kk, rci, rcj, kk, cs, cd);
        }
        __syncthreads();
        if (in) {
#pragma unroll
            for (int t = 0; t < TZ; ++t)
                if (t < nz) {
                    const int k = zb + t, idx = i + n0 * j + plane * k;
                    const T dc = sd[t + Z0][ty + 1][tx + 1];
                    T Ad;
                    if (plain) {
                        // every face carries cu: A d = cu (sum of the 2n neighbours - 2n d)
                        T nb = (sd[t + Z0][ty + 1][tx + 2] + sd[t + Z0][ty + 1][tx]) +
                               (sd[t + Z0][ty + 2][tx + 1] + sd[t + Z0][ty][tx + 1]);
                        if (NDIM == 3) nb += sd[t + 2 * Z0][ty + 1][tx + 1] + sd[t][ty + 1][tx + 1];
                        Ad = L.cu * (nb - T(2 * NDIM) * dc);
                    } else {
                        T cp[3], cm[3];
                        coefs<T, NDIM>(L, uni, i, j, k, idx, cp, cm);
                        Ad = cp[0] * (sd[t + Z0][ty + 1][tx + 2] - dc) - cm[0] * (dc - sd[t + Z0][ty + 1][tx]) +
                             cp[1] * (sd[t + Z0][ty + 2][tx + 1] - dc) - cm[1] * (dc - sd[t + Z0][ty][tx + 1]);
                        if (NDIM == 3)
                            Ad += cp[2] * (sd[t + 2 * Z0][ty + 1][tx + 1] - dc) - cm[2] * (dc - sd[t][ty + 1][tx + 1]);
                    }
                    dnew[idx] = dc;
                    q[idx] = Ad;
                    acc[0] += dc * Ad;
                }
        }
    });
    double out[1];
    if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_Q], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) S->alpha[lev] = out[0] != 0.0 ? S->rho[lev] / out[0] : 0.0;
}
template <typename T, int NDIM, bool FIRST>
__global__ void __launch_bounds__(256, 4) k_pcg_dq(LevelD<T> L, const T *dold, T *dnew,
                                                   DevScalars *S, double *part, int lev) {
    pcg_dq_run<T, NDIM>(L, dold, dnew, S, part, lev, FIRST);
}

// PCG start after the coarse correction: x = P x_c (injection), s = r - A x,
// rho = <s, D^-1 s> (the first search direction D^-1 s is formed by k_pcg_dq).
template <typename T, int NDIM>
__device__ __forceinline__ void pcg_init_run(const LevelD<T> &L, const GridD &gc, const T *xc, DevScalars *S,
                                             double *part, int lev) {
    const GridD &g = L.g;
    T acc[1] = {T(0)};
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const Col c = column(g, x0, y0);
        if (!c.in) return;
        // injection: the operand at a fine cell is its parent's coarse value
        const int ci = c.i >> 1, cj = c.j >> 1;
        const int cxm = ((c.i + c.oxm) >> 1) - ci, cxp = ((c.i + c.oxp) >> 1) - ci;
        const int cym = (((c.j + c.oym / g.n[0]) >> 1) - cj) * gc.n[0];
        const int cyp = (((c.j + c.oyp / g.n[0]) >> 1) - cj) * gc.n[0];
        const int cplane = gc.n[0] * gc.n[1];
        const int cbase = ci + gc.n[0] * cj;
        const bool pz = g.per[2] != 0;
        const int zb = NDIM == 3 ? z0 : 0, ze = NDIM == 3 ? min(z0 + MT<NDIM>::TZ, g.n[2]) : 1;
        constexpr int TZ = MT<NDIM>::TZ;
        constexpr int PZ = NDIM == 3 ? TZ + 2 : 1;
        // uniform tile away from every non-periodic domain face: every cell
        // has 2n faces of coefficient cu
        const bool plain = uni && (g.per[0] || (x0 > 0 && x0 + 32 < g.n[0])) &&
                           (g.per[1] || (y0 > 0 && y0 + 8 < g.n[1])) && (NDIM == 2 || pz || (zb > 0 && ze < g.n[2]));
        const T idc = T(-1) / (T(2 * NDIM) * L.cu);
        const T *__restrict__ rr = L.r;
        const T *__restrict__ id = L.invD;
        const T *__restrict__ xcr = xc;
        // every load of the column first: r and 1/D of its cells, the parent
        // value of fine planes zb-1 .. zb+TZ, and the parent of the x and of
        // the y neighbour that has another parent (the other side of each
        // pair shares the cell's parent: at most one offset is nonzero)
        const int cxn = cxm ? cxm : cxp, cyn = cym ? cym : cyp;
        T rv[TZ], iv[TZ], pv[PZ], xn[TZ], yn[TZ];
#pragma unroll
        for (int t = 0; t < PZ; ++t) {
            const int kf = NDIM == 3 ? edge_idx(zb - 1 + t, g.n[2], pz) : 0;
            if (NDIM == 2 || zb - 1 + t <= ze) pv[t] = xcr[cbase + cplane * (kf >> 1)];
        }
#pragma unroll
        for (int t = 0; t < TZ; ++t)
            if (zb + t < ze) {
                const int idx = c.i + g.n[0] * (c.j + g.n[1] * (zb + t));
                rv[t] = rr[idx];
                iv[t] = plain ? idc : id[idx];
                const int cb = cbase + cplane * (NDIM == 3 ? ((zb + t) >> 1) : 0);
                xn[t] = cxn ? xcr[cb + cxn] : T(0);
                yn[t] = cyn ? xcr[cb + cyn] : T(0);
            }
#pragma unroll
        for (int t = 0; t < TZ; ++t) {
            const int k = zb + t;
            if (k >= ze) break;
            const int idx = c.i + g.n[0] * (c.j + g.n[1] * k);
            const T x0v = pv[t + (NDIM == 3 ? 1 : 0)];
            L.x[idx] = x0v;
            const T iD = iv[t];
            T s = T(0);
            if (iD != T(0)) {
                const T vxm = cxm ? xn[t] : x0v, vxp = cxp ? xn[t] : x0v;
                const T vym = cym ? yn[t] : x0v, vyp = cyp ? yn[t] : x0v;
                T Ax;
                if (plain) {
                    // every face carries cu: A x = cu (sum of the 2n neighbours - 2n x)
                    T nb = (vxp + vxm) + (vyp + vym);
                    if (NDIM == 3) nb += pv[t + 2] + pv[t];
                    Ax = L.cu * (nb - T(2 * NDIM) * x0v);
                } else {
                    T cp[3], cm[3];
                    coefs<T, NDIM>(L, uni, c.i, c.j, k, idx, cp, cm);
                    Ax = cp[0] * (vxp - x0v) - cm[0] * (x0v - vxm) + cp[1] * (vyp - x0v) - cm[1] * (x0v - vym);
                    if (NDIM == 3) Ax += cp[2] * (pv[t + 2] - x0v) - cm[2] * (x0v - pv[t]);
                }
                s = rv[t] - Ax;
            }
            L.s[idx] = s;
            acc[0] += s * (iD * s);
        }
    });
    double out[1];
    if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_INIT], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) S->rho[lev] = out[0];
}
template <typename T, int NDIM>
__global__ void __launch_bounds__(256, 3) k_pcg_initm(LevelD<T> L, GridD gc, const T *xc, DevScalars *S, double *part,
                                                   int lev) {
    pcg_init_run<T, NDIM>(L, gc, xc, S, part, lev);
}
