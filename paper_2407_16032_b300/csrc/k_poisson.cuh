// k_poisson.cuh -- projection and geometric multigrid kernels.
//
// Sec. 2: the velocity is made divergence-free by a pressure projection whose
// variable-coefficient Poisson equation is solved by geometric multigrid;
// Sec. 3: the coefficients are c (face mu0) and the gradient update is
// u[I,a] -= c[I,a] (p[I] - p[I-e_a]);  Sec. 4.2: the multigrid smoother is a
// preconditioned conjugate gradient.
//
//   (A p)[I] = sum_a c_a[I+e_a](p[I+e_a]-p[I]) - c_a[I](p[I]-p[I-e_a])
//
// Layout and mapping: every level is swept in tiles of 32 x 8 (x TZ) cells, one
// 32x8 thread block per tile (grid-stride over tiles), so neighbour offsets are
// +-1, +-n0, +-n0*n1 with wrap-around only on the domain edge. A per-tile flag
// marks tiles whose faces (and those of a one-cell halo) all carry the level's
// fluid coefficient cu (or 0 on the domain boundary): there c and 1/D are
// formed from the position instead of being loaded.
//
// Precision: stencils and smoothing in the working type T. The refinement
// pressure is an unevaluated pair p = ph + pl of T values (double-T); its
// residual is evaluated with exact differences (two-sum) and exact products
// (FMA) wherever the coefficients vary, and by the second difference of exact
// hi-part differences where they are uniform. Norms and dot products are
// combined in double across warps and blocks; the coarsest level is solved in
// double.
#pragma once
#include "wl_common.cuh"

template <int NDIM> struct MT {
    static constexpr int TX = 32, TY = 8, TZ = NDIM == 3 ? 8 : 1;
};

struct Tiles {
    int ntx, nty, ntz, nt;
};

inline Tiles tiles_of(const GridD &g, int TZ) {
    Tiles t;
    t.ntx = (g.n[0] + 31) / 32;
    t.nty = (g.n[1] + 7) / 8;
    t.ntz = (g.n[2] + TZ - 1) / TZ;
    t.nt = t.ntx * t.nty * t.ntz;
    return t;
}

template <typename T> struct LevelD {
    GridD g;
    const T *c[3];
    T *invD;
    T *x, *r, *s, *q;
    T *d[2];
    const unsigned char *tflag;
    T cu;    // fluid face coefficient of this level
    T iduni; // 1/D of every cell when the level has no body and only periodic axes, else 0
    Tiles tl;
};

// Sweep all cells of a level tile by tile; f(i, j, k, idx, uniform_tile).
template <int NDIM, typename F>
__device__ __forceinline__ void for_cells(const GridD &g, const Tiles &tl, const unsigned char *tflag, F &&f) {
    for (int t = blockIdx.x; t < tl.nt; t += gridDim.x) {
        const int bx = t % tl.ntx, rr = t / tl.ntx;
        const int by = rr % tl.nty, bz = rr / tl.nty;
        const bool uni = tflag ? tflag[t] != 0 : false;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y;
        if (i >= g.n[0] || j >= g.n[1]) continue;
#pragma unroll
        for (int kk = 0; kk < MT<NDIM>::TZ; ++kk) {
            const int k = bz * MT<NDIM>::TZ + kk;
            if (k >= g.n[2]) break;
            const long long idx = (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
            f(i, j, k, idx, uni);
        }
    }
}

// A half-open box of cells of a level (lo <= index < hi on every axis).
struct CellBox {
    int lo[3], hi[3];
};

// Sweep the cells of a box, by the tiles of the level that meet it;
// f(i, j, k, idx).
template <int NDIM, typename F>
__device__ __forceinline__ void for_box_cells(const GridD &g, const CellBox &b, F &&f) {
    constexpr int TZ = MT<NDIM>::TZ;
    const int t0x = b.lo[0] / 32, t0y = b.lo[1] / 8, t0z = b.lo[2] / TZ;
    const int nx = (b.hi[0] + 31) / 32 - t0x, ny = (b.hi[1] + 7) / 8 - t0y, nz = (b.hi[2] + TZ - 1) / TZ - t0z;
    for (int q = blockIdx.x; q < nx * ny * nz; q += gridDim.x) {
        const int bx = t0x + q % nx, rr = q / nx;
        const int by = t0y + rr % ny, bz = t0z + rr / ny;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y;
        if (i < b.lo[0] || i >= b.hi[0] || j < b.lo[1] || j >= b.hi[1]) continue;
        for (int kk = 0; kk < TZ; ++kk) {
            const int k = bz * TZ + kk;
            if (k < b.lo[2]) continue;
            if (k >= b.hi[2]) break;
            f(i, j, k, (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k));
        }
    }
}

// The cells of box b as (tile, plane) work items, one 32 x 8 block each (a
// block per plane rather than per column: 8 times the blocks of
// for_box_cells, for work that is heavy per cell and a box that holds few
// tiles).
template <int NDIM, typename F>
__device__ __forceinline__ void for_box_planes(const GridD &g, const CellBox &b, F &&f) {
    constexpr int TZ = MT<NDIM>::TZ;
    const int t0x = b.lo[0] / 32, t0y = b.lo[1] / 8, t0z = b.lo[2] / TZ;
    const int nx = (b.hi[0] + 31) / 32 - t0x, ny = (b.hi[1] + 7) / 8 - t0y, nz = (b.hi[2] + TZ - 1) / TZ - t0z;
    for (int q = blockIdx.x; q < nx * ny * nz * TZ; q += gridDim.x) {
        const int tq = q / TZ, kk = q % TZ;
        const int bx = t0x + tq % nx, rr = tq / nx;
        const int by = t0y + rr % ny, bz = t0z + rr / ny;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y, k = bz * TZ + kk;
        if (i < b.lo[0] || i >= b.hi[0] || j < b.lo[1] || j >= b.hi[1] || k < b.lo[2] || k >= b.hi[2]) continue;
        f(i, j, k, (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k));
    }
}

// Walk the tiles of a level: body(x0, y0, z0, uniform) for each tile.
template <int NDIM, typename F>
__device__ __forceinline__ void for_tiles(const Tiles &tl, const unsigned char *tflag, F &&body) {
    for (int t = blockIdx.x; t < tl.nt; t += gridDim.x) {
        const int bx = t % tl.ntx, rr = t / tl.ntx;
        const int by = rr % tl.nty, bz = rr / tl.nty;
        body(bx * 32, by * 8, bz * MT<NDIM>::TZ, tflag ? tflag[t] != 0 : false);
    }
}

// Neighbour indices and face coefficients of cell (i,j,k) = idx. In uniform
// tiles the coefficients come from the position (cu, or 0 on a non-periodic
// domain face); elsewhere they are loaded.
template <typename T, int NDIM>
__device__ __forceinline__ void nb_setup(const LevelD<T> &L, bool uni, int i, int j, int k, long long idx,
                                         long long (&ip)[3], long long (&im)[3], T (&cp)[3], T (&cm)[3]) {
    const int I[3] = {i, j, k};
    const long long st[3] = {1, (long long)L.g.n[0], (long long)L.g.n[0] * L.g.n[1]};
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        const int N = L.g.n[a];
        const bool top = I[a] == N - 1, bot = I[a] == 0, per = L.g.per[a] != 0;
        ip[a] = top ? (per ? idx - (long long)(N - 1) * st[a] : idx) : idx + st[a];
        im[a] = bot ? (per ? idx + (long long)(N - 1) * st[a] : idx) : idx - st[a];
        if (uni) {
            cp[a] = (top && !per) ? T(0) : L.cu;
            cm[a] = (bot && !per) ? T(0) : L.cu;
        } else {
            cp[a] = (top && !per) ? T(0) : L.c[a][ip[a]];
            cm[a] = L.c[a][idx];
        }
    }
}

// 1/D of a cell of a uniform tile (all faces cu except non-periodic domain faces).
template <typename T, int NDIM>
__device__ __forceinline__ T invd_uniform(const LevelD<T> &L, int i, int j, int k) {
    const int I[3] = {i, j, k};
    int nf = 0;
#pragma unroll
    for (int a = 0; a < NDIM; ++a) {
        if (!L.g.per[a]) nf += (I[a] == 0) + (I[a] == L.g.n[a] - 1);
    }
    const int faces = 2 * NDIM - nf;
    return faces > 0 ? T(-1) / (T(faces) * L.cu) : T(0);
}

template <typename T, int NDIM>
__device__ __forceinline__ T invd_at(const LevelD<T> &L, bool uni, int i, int j, int k, long long idx) {
    return uni ? invd_uniform<T, NDIM>(L, i, j, k) : L.invD[idx];
}

// ------------------------------------------------------------------ set-up
// Inverse Jacobi diagonal 1/D, D = -sum of the 2n face coefficients (0 -> 0);
// counts active rows (D != 0) into S->nact when COUNT.
// On the cells of box b only; with COUNT, S->nact = active rows of the box +
// `outside` (every cell outside the box being active).
template <typename T, int NDIM, bool COUNT>
__global__ void __launch_bounds__(256) k_invd(LevelD<T> L, CellBox b, double outside, DevScalars *S, double *part) {
    T cnt[1] = {T(0)};
    for_box_cells<NDIM>(L.g, b, [&](int i, int j, int k, long long idx) {
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, false, i, j, k, idx, ip, im, cp, cm);
        T D = T(0);
#pragma unroll
        for (int a = 0; a < NDIM; ++a) D -= cp[a] + cm[a];
        L.invD[idx] = D != T(0) ? T(1) / D : T(0);
        if (COUNT && D != T(0)) cnt[0] += T(1);
    });
    if (COUNT) {
        double out[1];
        if (grid_reduce<1, false, T>(cnt, part, &S->counters[RS_INVD], out))
            if (threadIdx.x == 0 && threadIdx.y == 0) S->nact = out[0] + outside;
    }
}

// Set the flags of the tiles that meet box b to 1 (uniform, before k_tileflags).
template <int NDIM>
__global__ void k_tileflag_reset(Tiles tl, CellBox b, unsigned char *flags) {
    constexpr int TZ = MT<NDIM>::TZ;
    const int t0x = b.lo[0] / 32, t0y = b.lo[1] / 8, t0z = b.lo[2] / TZ;
    const int nx = (b.hi[0] + 31) / 32 - t0x, ny = (b.hi[1] + 7) / 8 - t0y, nz = (b.hi[2] + TZ - 1) / TZ - t0z;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx * ny * nz; q += gridDim.x * blockDim.x) {
        const int bx = t0x + q % nx, rr = q / nx;
        flags[bx + tl.ntx * ((t0y + rr % ny) + tl.nty * (t0z + rr / ny))] = 1;
    }
}

// Tile flags: clear the flag of every tile whose cells or one-cell halo have a
// face coefficient different from the uniform pattern (flags preset to 1).
// Scans the cells of box b (the other cells being uniform).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_tileflags(LevelD<T> L, CellBox b, unsigned char *flags) {
    for_box_cells<NDIM>(L.g, b, [&](int i, int j, int k, long long idx) {
        long long ip[3], im[3];
        T cp[3], cm[3], up[3], um[3];
        nb_setup<T, NDIM>(L, false, i, j, k, idx, ip, im, cp, cm);
        nb_setup<T, NDIM>(L, true, i, j, k, idx, ip, im, up, um);
        bool ok = true;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) ok = ok && cp[a] == up[a] && cm[a] == um[a];
        if (ok) return;
        const int I[3] = {i, j, k};
        const int TZ = MT<NDIM>::TZ;
        for (int dz = (NDIM == 3 ? -1 : 0); dz <= (NDIM == 3 ? 1 : 0); ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int J[3] = {I[0] + dx, I[1] + dy, I[2] + dz};
                    bool skip = false;
                    for (int a = 0; a < NDIM; ++a) {
                        if (J[a] < 0 || J[a] >= L.g.n[a]) {
                            if (L.g.per[a]) J[a] = wrapi(J[a], L.g.n[a]);
                            else skip = true;
                        }
                    }
                    if (skip) continue;
                    const int t = (J[0] / 32) + L.tl.ntx * ((J[1] / 8) + L.tl.nty * (J[2] / TZ));
                    flags[t] = 0;
                }
    });
}

// Coarse coefficients: half the sum of the 2^(n-1) fine faces on each coarse face.
// On the coarse cells of box b.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_coarsen_c(GridD gf, CVec3P<T> cf, LevelD<T> C, CellBox b, Vec3P<T> cc) {
    for_box_cells<NDIM>(C.g, b, [&](int i, int j, int k, long long idx) {
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            T s = T(0);
            for (int oz = 0; oz < (NDIM == 3 ? 2 : 1); ++oz)
                for (int oy = 0; oy < 2; ++oy)
                    for (int ox = 0; ox < 2; ++ox) {
                        const int o[3] = {ox, oy, oz};
                        if (o[a] != 0) continue;
                        s += cf.p[a][lin3(gf, 2 * i + ox, 2 * j + oy, 2 * k + oz)];
                    }
            cc.p[a][idx] = T(0.5) * s;
        }
    });
}

// --------------------------------------------------------- right-hand side
// b = div(u) / (w dt) (Sec. 2 projection) and its sum / sum of squares over
// active rows -> mean and |b - mean|.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e);

template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_div(LevelD<T> L, CVec3P<T> u, const T *ue, T inv_wdt, T *b, T *bl,
                                             DevScalars *S, double *part) {
    constexpr int TZ = MT<NDIM>::TZ;
    const GridD &g = L.g;
    T acc[2] = {T(0), T(0)};
    const T *__restrict__ ux = u.p[0], *__restrict__ uy = u.p[1], *__restrict__ uz = u.p[2];
    const T *__restrict__ uep = ue;
    const T *__restrict__ iDp = L.invD;
    T *__restrict__ bo = b, *__restrict__ blo = bl;
    const long long plane = (long long)g.n[0] * g.n[1];
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
        if (i >= g.n[0] || j >= g.n[1]) return;
        const int zb = NDIM == 3 ? z0 : 0, nz = NDIM == 3 ? min(TZ, g.n[2] - z0) : 1;
        const long long base = i + (long long)g.n[0] * j;
        // upper faces: the next cell, the periodic image, or the boundary value
        // (U_a, or the exit plane for u_x)
        const bool xin = i + 1 < g.n[0], yin = j + 1 < g.n[1];
        const long long ox = xin ? 1 : (g.per[0] ? -(long long)(g.n[0] - 1) : 0);
        const long long oy = yin ? g.n[0] : (g.per[1] ? -(long long)(g.n[1] - 1) * g.n[0] : 0);
        const bool xb = !xin && !g.per[0], yb = !yin && !g.per[1];
        // every load of the column first
        T vx[TZ], vxp[TZ], vy[TZ], vyp[TZ], vz[TZ + 1], iv[TZ];
#pragma unroll
        for (int t = 0; t < TZ; ++t)
            if (t < nz) {
                const long long idx = base + plane * (zb + t);
                vx[t] = ux[idx];
                vxp[t] = xb ? (g.exit_x ? uep[j + (long long)g.n[1] * (zb + t)] : (T)g.U[0]) : ux[idx + ox];
                vy[t] = uy[idx];
                vyp[t] = yb ? (T)g.U[1] : uy[idx + oy];
                if (NDIM == 3) vz[t] = uz[idx];
                iv[t] = uni ? T(1) : iDp[idx];
            }
        if (NDIM == 3) {
            const int kt = zb + nz;
            vz[nz < TZ ? nz : TZ] = kt < g.n[2] ? uz[base + plane * kt] : (g.per[2] ? uz[base] : (T)g.U[2]);
        }
#pragma unroll
        for (int t = 0; t < TZ; ++t)
            if (t < nz) {
                const long long idx = base + plane * (zb + t);
                // divergence as an unevaluated pair (exact face differences,
                // two-sum accumulation over the axes in order), scaled by 1/(w dt)
                const T up[3] = {vxp[t], vyp[t], NDIM == 3 ? vz[t + 1] : T(0)};
                const T lo[3] = {vx[t], vy[t], NDIM == 3 ? vz[t] : T(0)};
                T sh = T(0), sl = T(0);
#pragma unroll
                for (int a = 0; a < NDIM; ++a) {
                    T d, de, s2, e2;
                    two_sum(up[a], -lo[a], d, de);
                    two_sum(sh, d, s2, e2);
                    sh = s2;
                    sl += e2 + de;
                }
                T h = sh + sl;
                T l = sl - (h - sh);
                const T bh = h * inv_wdt;
                const T blo_ = fma(h, inv_wdt, -bh) + l * inv_wdt;
                const T sv = bh + blo_;
                bo[idx] = sv;
                blo[idx] = blo_ - (sv - bh);
                if (iv[t] != T(0)) { acc[0] += sv; acc[1] += sv * sv; }
            }
    });
    double out[2];
    if (grid_reduce<2, false, T>(acc, part, &S->counters[RS_DIV], out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double n = S->nact > 0 ? S->nact : 1.0;
            S->bsum = out[0];
            S->bsq = out[1];
            S->bmean = out[0] / n;
            const double v = out[1] - out[0] * out[0] / n;
            S->bnorm = sqrt(v > 0 ? v : 0.0);
            if (!(out[1] == out[1]) || out[1] > 1e300) S->status |= 1;
        }
    }
}

// Statistics of a given right-hand side b over active rows.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_bstats(LevelD<T> L, const T *b, DevScalars *S, double *part) {
    T acc[2] = {T(0), T(0)};
    for_cells<NDIM>(L.g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (uni || L.invD[idx] != T(0)) { const T v = b[idx]; acc[0] += v; acc[1] += v * v; }
    });
    double out[2];
    if (grid_reduce<2, false, T>(acc, part, &S->counters[RS_DIV], out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const double n = S->nact > 0 ? S->nact : 1.0;
            S->bsum = out[0];
            S->bsq = out[1];
            S->bmean = out[0] / n;
            const double v = out[1] - out[0] * out[0] / n;
            S->bnorm = sqrt(v > 0 ? v : 0.0);
            if (!(out[1] == out[1]) || out[1] > 1e300) S->status |= 1;
        }
    }
}

// ---------------------------------------------------- refinement residual
// Exact pair arithmetic on T (two-sum, FMA two-product).
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// c * (pN - p0) as an unevaluated pair, from the pairs (hN, lN), (h0, l0).
template <typename T>
__device__ __forceinline__ void face_term(T hN, T lN, T h0, T l0, T c, T &th, T &tl) {
    T s, e;
    two_sum(hN, -h0, s, e);
    e += lN - l0;
    const T dh = s + e;
    const T dl = e - (dh - s);
    th = c * dh;
    tl = fma(c, dh, -th) + c * dl;
}

// Restriction: coarse r = sum of the 2^n fine children.
template <typename T, int NDIM>
__device__ __forceinline__ void restrict_run(const GridD &gf, const T *rf, const LevelD<T> &C) {
    for_cells<NDIM>(C.g, C.tl, nullptr, [&](int i, int j, int k, long long idx, bool) {
        T s = T(0);
        for (int oz = 0; oz < (NDIM == 3 ? 2 : 1); ++oz)
            for (int oy = 0; oy < 2; ++oy) {
                const long long base = lin3(gf, 2 * i, 2 * j + oy, 2 * k + oz);
                s += rf[base] + rf[base + 1];
            }
        C.r[idx] = s;
    });
}
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_restrict(GridD gf, const T *rf, LevelD<T> C) {
    restrict_run<T, NDIM>(gf, rf, C);
}

// Parent (injection) index of the fine cell (i,j,k) offset by o along axis a,
// wrapped on periodic axes, clamped otherwise (its coefficient is 0 there).
__device__ __forceinline__ long long parent_off(const GridD &gf, const GridD &gc, int i, int j, int k, int a, int o) {
    int I[3] = {i, j, k};
    I[a] += o;
    if (I[a] < 0) I[a] = gf.per[a] ? gf.n[a] - 1 : 0;
    if (I[a] >= gf.n[a]) I[a] = gf.per[a] ? 0 : gf.n[a] - 1;
    return lin3(gc, I[0] >> 1, I[1] >> 1, gf.ndim == 3 ? (I[2] >> 1) : 0);
}

// PCG step part 2: x += alpha d; s -= alpha q; rho' = <s, D^-1 s>; beta = rho'/rho.
// On the last iteration only x is updated; on the fine level the correction
// is added straight into the refinement pressure (ph, pl) instead.
// Purely elementwise: a linear sweep in 16-byte vectors.
template <typename T> struct V16;
template <> struct V16<float> { typedef float4 type; static constexpr int n = 4; };
template <> struct V16<double> { typedef double2 type; static constexpr int n = 2; };

template <typename T, bool LAST, bool FINE>
__device__ __forceinline__ void pcg_u_elem(T &x, T d, T &s, T q, T iD, T &ph, T &pl, T alpha, T &acc) {
    const T xn = x + alpha * d;
    if (LAST && FINE) {
        T sh, err;
        two_sum(ph, xn, sh, err);
        const T lo = pl + err;
        const T hi = sh + lo;
        ph = hi;
        pl = lo - (hi - sh);
    } else {
        x = xn;
    }
    if (!LAST) {
        s = s - alpha * q;
        acc += s * iD * s;
    }
}

template <typename T, bool LAST, bool FINE>
__device__ __forceinline__ void pcg_u_run(const LevelD<T> &L, const T *dcur, T *ph, T *pl, DevScalars *S,
                                          double *part, int lev) {
    typedef typename V16<T>::type VT;
    constexpr int W = V16<T>::n;
    const T alpha = (T)S->alpha[lev];
    T acc[1] = {T(0)};
    const long long n = L.g.nc;
    const long long nv = (n % W == 0) ? n / W : 0;
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const long long stride = (long long)gridDim.x * nthr;
    const long long t0 = blockIdx.x * (long long)nthr + tid;
    const T idc = L.iduni;
    for (long long v = t0; v < nv; v += stride) {
        VT x = ((VT *)L.x)[v], d = ((const VT *)dcur)[v], s = ((VT *)L.s)[v], q = ((const VT *)L.q)[v];
        VT iD;
        if (idc != T(0) || LAST) {
            // (a constant diagonal; the last update does not use it)
            T *ie = (T *)&iD;
#pragma unroll
            for (int e = 0; e < W; ++e) ie[e] = idc;
        } else {
            iD = ((const VT *)L.invD)[v];
        }
        VT h, l;
        if (LAST && FINE) { h = ((VT *)ph)[v]; l = ((VT *)pl)[v]; }
        T *xe = (T *)&x, *se = (T *)&s, *he = (T *)&h, *le = (T *)&l;
        const T *de = (const T *)&d, *qe = (const T *)&q, *ie = (const T *)&iD;
#pragma unroll
        for (int e = 0; e < W; ++e) pcg_u_elem<T, LAST, FINE>(xe[e], de[e], se[e], qe[e], ie[e], he[e], le[e], alpha, acc[0]);
        if (LAST && FINE) { ((VT *)ph)[v] = h; ((VT *)pl)[v] = l; }
        else ((VT *)L.x)[v] = x;
        if (!LAST) ((VT *)L.s)[v] = s;
    }
    if (nv == 0)
        for (long long e = t0; e < n; e += stride) {
            T dummyh = T(0), dummyl = T(0);
            T *hp = (LAST && FINE) ? &ph[e] : &dummyh, *lp = (LAST && FINE) ? &pl[e] : &dummyl;
            pcg_u_elem<T, LAST, FINE>(L.x[e], dcur[e], L.s[e], L.q[e], L.invD[e], *hp, *lp, alpha, acc[0]);
        }
    if (!LAST) {
        double out[1];
        if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_U], out))
            if (tid == 0) {
                const double rho = S->rho[lev];
                S->beta[lev] = rho != 0.0 ? out[0] / rho : 0.0;
                S->rho[lev] = out[0];
            }
    }
}

template <typename T, bool LAST, bool FINE>
__global__ void __launch_bounds__(256) k_pcg_u(LevelD<T> L, const T *dcur, T *ph, T *pl, DevScalars *S, double *part,
                                               int lev, int it) {
    pcg_u_run<T, LAST, FINE>(L, dcur, ph, pl, S, part, lev);
}

// The weak rows themselves: the active level-0 cells of the listed tiles whose
// face coefficients sum to less than cut, appended to wlist (in no
// particular order; each row's update below is independent of the order).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_weak_list(LevelD<T> L, double cut, const int *tlist, const unsigned *tcount,
                                                   int *wlist, unsigned *wcount) {
    const GridD &g = L.g;
    // work items: (listed non-uniform tile, plane of the tile), a 32 x 8 block each
    const int nb = (int)*tcount * MT<NDIM>::TZ;
    for (int q = blockIdx.x; q < nb; q += gridDim.x) {
        const int t = tlist[q / MT<NDIM>::TZ];
        const int bx = t % L.tl.ntx, rr = t / L.tl.ntx;
        const int by = rr % L.tl.nty, bz = rr / L.tl.nty;
        const int i = bx * 32 + threadIdx.x, j = by * 8 + threadIdx.y;
        const int k = bz * MT<NDIM>::TZ + q % MT<NDIM>::TZ;
        if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) continue;
        const long long idx = (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * k);
        if (L.invD[idx] == T(0)) continue;
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, false, i, j, k, idx, ip, im, cp, cm);
        double csum = 0.0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) csum += (double)cp[a] + (double)cm[a];
        if (csum > 0.0 && csum < cut) wlist[atomicAdd(wcount, 1u)] = (int)idx;
    }
}

// Weakly coupled rows after a solve. A row whose face coefficients sum to
// less than `cut` has its pressure fixed by the solve only to r / sum c, and r
// is bounded by the global residual norm, not by the row's own size; where the
// BDIM kernel weight is not zero such a row still enters the pressure force.
// A Gauss-Seidel update in double, p += r / A_II (A_II = -sum c) with
// r = (b - mean) - A p formed from the pairs, sets the row's residual to
// rounding and changes a neighbour's residual by c_f dp, at most |r|. Cells of
// one colour ((i + j + k) parity) read only the other colour, so an update is
// race-free and the result does not depend on the thread order. Level 0, over
// the rows k_weak_list collected.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_weak_rows(LevelD<T> L, const T *__restrict__ b, const T *__restrict__ bl,
                                                   T *ph, T *pl, const DevScalars *S, int colour, const int *wlist,
                                                   const unsigned *wcount) {
    const double bm = S->bmean;
    const GridD &g = L.g;
    const int nw = (int)*wcount;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw; e += gridDim.x * blockDim.x) {
        const long long idx = wlist[e];
        int i, j, k;
        decode(g, idx, i, j, k);
        if (((i + j + k) & 1) != colour) continue;
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, false, i, j, k, idx, ip, im, cp, cm);
        double csum = 0.0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) csum += (double)cp[a] + (double)cm[a];
        const double p0 = (double)ph[idx] + (double)pl[idx];
        double Ap = 0.0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            Ap += (double)cp[a] * (((double)ph[ip[a]] + (double)pl[ip[a]]) - p0);
            Ap += (double)cm[a] * (((double)ph[im[a]] + (double)pl[im[a]]) - p0);
        }
        const double r = (((double)b[idx] + (double)bl[idx]) - bm) - Ap;
        const double pn = p0 - r / csum;   // p += r / A_II, A_II = -csum
        const T h = (T)pn;
        ph[idx] = h;
        pl[idx] = (T)(pn - (double)h);
    }
}

// Single-level case: the coarse solve itself is the fine correction.
template <typename T>
__global__ void k_padd(GridD g, const T *x, T *ph, T *pl) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        T sh, err;
        two_sum(ph[idx], x[idx], sh, err);
        const T lo = pl[idx] + err;
        const T hi = sh + lo;
        ph[idx] = hi;
        pl[idx] = lo - (hi - sh);
    }
}

// One thread block, double-precision Jacobi-preconditioned CG on the mean-free
// part of a right-hand side over active rows (rows with a nonzero diagonal),
// A x = r - mean(r), from x = 0, until |s| <= rtol |s_0| or maxit iterations;
// the solution is made mean-free over active rows and written through the
// operator. Op supplies the problem:
//   long long n() const;                 number of cells
//   double invd(long long e) const;      1/D of row e (0: inactive row)
//   double rhs(long long e) const;       r[e]
//   double apply(const double *d, long long e) const;   (A d)[e]
//   void out(long long e, double x) const;              store x[e] (0 on inactive rows)
// Scratch: xs, ss, ds, qs, n doubles each. Returns |s| / |s_0| (0 if s_0 = 0)
// in every thread. Used by the coarsest multigrid level and by
// wl_coarse_solve_static, so both solve with the same arithmetic.
template <class Op>
__device__ __forceinline__ double block_pcg_solve(const Op &op, double *xs, double *ss, double *ds, double *qs,
                                                  int maxit, double rtol) {
    const long long n = op.n();
    __shared__ double sh[64];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    double v1[1], o1[1];
    double sr = 0.0, na = 0.0;
    for (long long e = tid; e < n; e += nt)
        if (op.invd(e) != 0.0) { sr += op.rhs(e); na += 1.0; }
    double v2[2] = {sr, na}, o2[2];
    block_reduce<2, false, double>(v2, o2, sh);
    if (tid == 0) { sh[40] = o2[0]; sh[41] = o2[1]; }
    __syncthreads();
    const double rmean = sh[41] > 0 ? sh[40] / sh[41] : 0.0, nact = sh[41];
    __syncthreads();
    double r0 = 0.0, rho = 0.0;
    for (long long e = tid; e < n; e += nt) {
        const double iD = op.invd(e);
        const double s = iD != 0.0 ? op.rhs(e) - rmean : 0.0;
        xs[e] = 0.0;  // scratch may hold an earlier solve: start from zero
        ss[e] = s;
        ds[e] = iD * s;
        rho += s * ds[e];
        r0 += s * s;
    }
    double v3[2] = {rho, r0}, o3[2];
    block_reduce<2, false, double>(v3, o3, sh);
    if (tid == 0) { sh[40] = o3[0]; sh[41] = o3[1]; }
    __syncthreads();
    rho = sh[40];
    const double rnorm0 = sqrt(sh[41]);
    double sn = rnorm0;
    __syncthreads();
    for (int it = 0; it < maxit && rho != 0.0 && sn > rtol * rnorm0; ++it) {
        double dq = 0.0;
        for (long long e = tid; e < n; e += nt) {
            const double Ad = op.apply(ds, e);
            qs[e] = Ad;
            dq += ds[e] * Ad;
        }
        v1[0] = dq;
        block_reduce<1, false, double>(v1, o1, sh);
        if (tid == 0) sh[40] = o1[0];
        __syncthreads();
        dq = sh[40];
        __syncthreads();
        if (dq == 0.0) break;
        const double alpha = rho / dq;
        double rn = 0.0, ss2 = 0.0;
        for (long long e = tid; e < n; e += nt) {
            xs[e] += alpha * ds[e];
            const double s = ss[e] - alpha * qs[e];
            ss[e] = s;
            rn += s * op.invd(e) * s;
            ss2 += s * s;
        }
        v3[0] = rn;
        v3[1] = ss2;
        block_reduce<2, false, double>(v3, o3, sh);
        if (tid == 0) { sh[40] = o3[0]; sh[41] = o3[1]; }
        __syncthreads();
        const double rho2 = sh[40];
        sn = sqrt(sh[41]);
        __syncthreads();
        const double beta = rho2 / rho;
        rho = rho2;
        for (long long e = tid; e < n; e += nt) ds[e] = op.invd(e) * ss[e] + beta * ds[e];
        __syncthreads();
    }
    double sx = 0.0;
    for (long long e = tid; e < n; e += nt)
        if (op.invd(e) != 0.0) sx += xs[e];
    v1[0] = sx;
    block_reduce<1, false, double>(v1, o1, sh);
    if (tid == 0) sh[40] = o1[0];
    __syncthreads();
    const double xm = nact > 0 ? sh[40] / nact : 0.0;
    for (long long e = tid; e < n; e += nt) op.out(e, op.invd(e) != 0.0 ? xs[e] - xm : 0.0);
    return rnorm0 > 0 ? sn / rnorm0 : 0.0;
}

// (A d)[e] of a level with lower-face coefficients c[a] (cell e's own lower
// face; the upper face is the next cell's, 0 at the top of a non-periodic
// axis; periodic axes wrap), in double.
template <typename T>
__device__ __forceinline__ double level_apply(const GridD &g, const T *const *c, const double *d, long long e) {
    const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    const long long q = e / g.n[0];
    const int I[3] = {(int)(e - q * g.n[0]), (int)(q % g.n[1]), (int)(q / g.n[1])};
    double Ad = 0.0;
    const double d0 = d[e];
    for (int a = 0; a < g.ndim; ++a) {
        const int N = g.n[a];
        const bool top = I[a] == N - 1, bot = I[a] == 0, per = g.per[a] != 0;
        const long long ip = top ? (per ? e - (long long)(N - 1) * st[a] : e) : e + st[a];
        const long long im = bot ? (per ? e + (long long)(N - 1) * st[a] : e) : e - st[a];
        const double cp = (top && !per) ? 0.0 : (double)c[a][ip];
        const double cm = (double)c[a][e];
        Ad += cp * (d[ip] - d0) - cm * (d0 - d[im]);
    }
    return Ad;
}

// Coarsest level: one block, Jacobi-PCG in double to 1e-12 relative or maxit;
// the mean-free solution is written to L.x. w: 4*nc doubles of scratch.
template <typename T>
struct CoarsestOp {
    LevelD<T> L;
    __device__ long long n() const { return L.g.nc; }
    __device__ double invd(long long e) const { return (double)L.invD[e]; }
    __device__ double rhs(long long e) const { return (double)L.r[e]; }
    __device__ double apply(const double *d, long long e) const { return level_apply<T>(L.g, L.c, d, e); }
    __device__ void out(long long e, double x) const { L.x[e] = (T)x; }
};
template <typename T>
__global__ void k_coarsest(LevelD<T> L, double *w, int maxit) {
    const long long n = L.g.nc;
    block_pcg_solve(CoarsestOp<T>{L}, w, w + n, w + 2 * n, w + 3 * n, maxit, 1e-12);
}

// Dense solution operator of the coarsest level, built on the device: block j
// solves A x = e_j - mean(e_j) (mean over active rows) by block_pcg_solve to
// 1e-13 and writes the mean-free x as column j of M (M[e * n + j]); columns of
// inactive rows come out zero. M is the active block of the inverse of the
// operator bordered by the mean constraint, as k_coarsest_dense expects. One
// block per column: the solves run side by side on the SMs. w: 4 n doubles of
// scratch per block.
template <typename T>
struct UnitColumnOp {
    LevelD<T> L;
    int j;
    double *M;
    __device__ long long n() const { return L.g.nc; }
    __device__ double invd(long long e) const { return (double)L.invD[e]; }
    __device__ double rhs(long long e) const { return e == j ? 1.0 : 0.0; }
    __device__ double apply(const double *d, long long e) const { return level_apply<T>(L.g, L.c, d, e); }
    __device__ void out(long long e, double x) const { M[e * L.g.nc + j] = x; }
};
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_operator(LevelD<T> L, double *M, double *w, int maxit) {
    const long long n = L.g.nc;
    double *wb = w + 4 * n * blockIdx.x;
    block_pcg_solve(UnitColumnOp<T>{L, (int)blockIdx.x, M}, wb, wb + n, wb + 2 * n, wb + 3 * n, maxit, 1e-13);
}

// Coarsest level by a precomputed dense solution operator (one block, FP64):
// x = M (r - mean r) over active rows, M the active block of the inverse of
// the operator bordered by the mean constraint, [A 1; 1^T 0]; x is made
// mean-free over active rows like the PCG solve's. M: n x n doubles, zero on
// inactive rows and columns.
template <typename T>
__global__ void k_coarsest_dense(LevelD<T> L, const double *__restrict__ M) {
    const int n = (int)L.g.nc;
    __shared__ double rr[512];
    __shared__ double sh[64];
    const int tid = threadIdx.x, nt = blockDim.x;
    double v2[2] = {0.0, 0.0}, o2[2];
    for (int e = tid; e < n; e += nt)
        if (L.invD[e] != T(0)) { v2[0] += (double)L.r[e]; v2[1] += 1.0; }
    block_reduce<2, false, double>(v2, o2, sh);
    if (tid == 0) { sh[40] = o2[0]; sh[41] = o2[1]; }
    __syncthreads();
    const double nact = sh[41], rmean = nact > 0 ? sh[40] / nact : 0.0;
    for (int e = tid; e < n; e += nt) rr[e] = L.invD[e] != T(0) ? (double)L.r[e] - rmean : 0.0;
    __syncthreads();
    double xs[2] = {0.0, 0.0};
    double sx = 0.0;
    for (int q = 0, e = tid; e < n; e += nt, ++q) {
        const double *row = M + (long long)e * n;
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc = fma(row[c], rr[c], acc);
        if (q < 2) xs[q] = acc;
        if (L.invD[e] != T(0)) sx += acc;
    }
    double v1[1] = {sx}, o1[1];
    block_reduce<1, false, double>(v1, o1, sh);
    if (tid == 0) sh[40] = o1[0];
    __syncthreads();
    const double xm = nact > 0 ? sh[40] / nact : 0.0;
    for (int q = 0, e = tid; e < n; e += nt, ++q) L.x[e] = L.invD[e] != T(0) ? (T)(xs[q] - xm) : T(0);
}

// ------------------------------------------------------------- projection
// Pressure-gradient update (Sec. 3 listing): u_a[I] -= w dt c_a[I] (p[I] - p[I-e_a]).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_grad(LevelD<T> L, const T *__restrict__ ph, const T *__restrict__ pl, T wdt,
                                              Vec3P<T> u) {
    constexpr int TZ = MT<NDIM>::TZ;
    constexpr int HB = NDIM == 3 ? 2 : 1;   // planes whose loads are issued together
    const GridD &g = L.g;
    T *__restrict__ ux = u.p[0], *__restrict__ uy = u.p[1], *__restrict__ uz = u.p[2];
    const long long plane = (long long)g.n[0] * g.n[1];
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int i = x0 + threadIdx.x, j = y0 + threadIdx.y;
        if (i >= g.n[0] || j >= g.n[1]) return;
        const int zb = NDIM == 3 ? z0 : 0, nz = NDIM == 3 ? min(TZ, g.n[2] - z0) : 1;
        const long long base = i + (long long)g.n[0] * j;
        // lower neighbours: the previous cell or the periodic image (a
        // non-periodic lower domain face has coefficient 0: no update)
        const long long om0 = i > 0 ? 1 : (long long)(g.n[0] - 1), om1 = j > 0 ? g.n[0] : (long long)(g.n[1] - 1) * g.n[0];
        const bool fx = i > 0 || g.per[0], fy = j > 0 || g.per[1];
        const long long sx = i > 0 ? -om0 : om0, sy = j > 0 ? -om1 : om1;
        for (int hb = 0; hb < nz; hb += HB) {
            T h0[HB], l0[HB], hx[HB], lx[HB], hy[HB], ly[HB], hz[HB], lz[HB], cx[HB], cy[HB], cz[HB];
            T vx[HB], vy[HB], vz[HB];
#pragma unroll
            for (int t = 0; t < HB; ++t)
                if (hb + t < nz) {
                    const int k = zb + hb + t;
                    const long long idx = base + plane * k;
                    h0[t] = ph[idx];
                    l0[t] = pl[idx];
                    vx[t] = ux[idx];
                    vy[t] = uy[idx];
                    if (NDIM == 3) vz[t] = uz[idx];
                    hx[t] = ph[idx + sx];
                    lx[t] = pl[idx + sx];
                    hy[t] = ph[idx + sy];
                    ly[t] = pl[idx + sy];
                    if (NDIM == 3) {
                        const long long km = k > 0 ? idx - plane : idx + plane * (g.n[2] - 1);
                        hz[t] = ph[km];
                        lz[t] = pl[km];
                    }
                    if (!uni) {
                        cx[t] = L.c[0][idx];
                        cy[t] = L.c[1][idx];
                        if (NDIM == 3) cz[t] = L.c[2][idx];
                    }
                }
#pragma unroll
            for (int t = 0; t < HB; ++t)
                if (hb + t < nz) {
                    const int k = zb + hb + t;
                    const long long idx = base + plane * k;
                    const bool fz = NDIM == 3 && (k > 0 || g.per[2]);
                    const T c0 = uni ? (fx ? L.cu : T(0)) : cx[t];
                    const T c1 = uni ? (fy ? L.cu : T(0)) : cy[t];
                    if (c0 != T(0)) ux[idx] = vx[t] - wdt * c0 * ((h0[t] - hx[t]) + (l0[t] - lx[t]));
                    if (c1 != T(0)) uy[idx] = vy[t] - wdt * c1 * ((h0[t] - hy[t]) + (l0[t] - ly[t]));
                    if (NDIM == 3) {
                        const T c2 = uni ? (fz ? L.cu : T(0)) : cz[t];
                        if (c2 != T(0)) uz[idx] = vz[t] - wdt * c2 * ((h0[t] - hz[t]) + (l0[t] - lz[t]));
                    }
                }
        }
    });
}

// Mean of the pressure over active rows -> S->pmean.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_pmean(LevelD<T> L, const T *ph, const T *pl, DevScalars *S, double *part) {
    T acc[2] = {T(0), T(0)};
    for_cells<NDIM>(L.g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (uni || L.invD[idx] != T(0)) { acc[0] += ph[idx]; acc[1] += pl[idx]; }
    });
    double out[2];
    if (grid_reduce<2, false, T>(acc, part, &S->counters[RS_PMEAN], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) S->pmean = S->nact > 0 ? (out[0] + out[1]) / S->nact : 0.0;
}

// Reported pressure: p - mean on active rows, 0 elsewhere (double).
template <typename T>
__global__ void k_pout(GridD g, const T *ph, const T *pl, const T *invD, const DevScalars *S, double *p) {
    const double pm = S->pmean;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x)
        p[idx] = invD[idx] != T(0) ? ((double)ph[idx] - pm) + (double)pl[idx] : 0.0;
}

// Warm start from doubles: split into (hi, lo).
template <typename T>
__global__ void k_pin(GridD g, const double *p, T *ph, T *pl) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.nc;
         idx += (long long)gridDim.x * blockDim.x) {
        const double v = p[idx];
        const T h = (T)v;
        ph[idx] = h;
        pl[idx] = (T)(v - (double)h);
    }
}
