// k_mg_march.cuh -- shared-memory z-marching 7-point stencils of the V-cycle.
//
// The operator is the variable-coefficient Poisson operator of the projection
// (Sec. 2, Sec. 3: u[I,i] -= c[I,i](p[I]-p[I-d(i)]) is its gradient half):
//   (A p)[I] = sum_a c_a[I+e_a](p[I+e_a]-p[I]) - c_a[I](p[I]-p[I-e_a]).
// Each 32x8 thread block owns a 32 x 8 x TZ tile. It stages the operand of the
// tile and a one-cell halo (ZC + 2 planes) in shared memory in one burst of
// independent coalesced loads, then computes ZC planes from it: every operand
// value is loaded, or formed (the PCG search direction d = D^-1 s + beta
// d_prev), once per tile and read by its seven stencil users from shared
// memory. The domain edge wraps (periodic, any distance) or clamps (the
// coefficient there is 0).
#pragma once
#include "k_poisson.cuh"

template <int NDIM> struct MW {
    static constexpr int TX = 32, TY = 8, TZ = MT<NDIM>::TZ;
    static constexpr int WX = TX + 2, WY = TY + 2, WN = WX * WY;
};
// Planes computed per slab load (the slab holds ZC + 2 planes in 3D): all of
// a tile's 8 planes in single precision, half of them in double.
template <int NDIM, typename T> struct MZ {
    static constexpr int ZC = NDIM == 3 ? (sizeof(T) == 4 ? MT<NDIM>::TZ : MT<NDIM>::TZ / 2) : 1;
    static constexpr int NPL = NDIM == 3 ? ZC + 2 : 1;
};

// Index along an axis of N cells: periodic axes wrap (any distance: the
// window is wider than small coarse levels), others clamp.
__device__ __forceinline__ int edge_idx(int v, int N, bool per) {
    if (v >= 0 && v < N) return v;
    if (per) {
        const int r = v % N;
        return r < 0 ? r + N : r;
    }
    return v < 0 ? 0 : N - 1;
}

// Load the slab of planes zs-1 .. zs+ZC (3D; the single plane in 2D) of the
// tile at (x0, y0) with its one-cell xy halo: slab[e] = f(global index). All
// loads of the slab are independent, so a block keeps them all in flight.
template <int NDIM, typename T, typename F>
__device__ __forceinline__ void load_slab(T *slab, const GridD &g, int x0, int y0, int zs, F &&f) {
    using W = MW<NDIM>;
    constexpr int NPL = MZ<NDIM, T>::NPL;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    for (int e = tid; e < NPL * W::WN; e += 256) {
        const int pl = e / W::WN, rem = e - pl * W::WN;
        const int ly = rem / W::WX, lx = rem - ly * W::WX;
        const int gx = edge_idx(x0 + lx - 1, g.n[0], g.per[0] != 0);
        const int gy = edge_idx(y0 + ly - 1, g.n[1], g.per[1] != 0);
        const int gz = NDIM == 3 ? edge_idx(zs - 1 + pl, g.n[2], g.per[2] != 0) : 0;
        slab[e] = f(gx + g.n[0] * (gy + g.n[1] * gz));
    }
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

// The six neighbours of the window centre (tx, ty) of plane slots pm/pc/pp.
template <int NDIM, typename T>
struct Nb6 {
    T c, xm, xp, ym, yp, zm, zp;
};
template <int NDIM, typename T>
__device__ __forceinline__ Nb6<NDIM, T> nb6(const T *pm, const T *pc, const T *pp) {
    using W = MW<NDIM>;
    const int o = (threadIdx.y + 1) * W::WX + threadIdx.x + 1;
    Nb6<NDIM, T> r;
    r.c = pc[o];
    r.xm = pc[o - 1];
    r.xp = pc[o + 1];
    r.ym = pc[o - W::WX];
    r.yp = pc[o + W::WX];
    if (NDIM == 3) { r.zm = pm[o]; r.zp = pp[o]; } else { r.zm = r.zp = T(0); }
    return r;
}

// Walk the tiles of a level: body(x0, y0, z0, uniform) for each tile.
template <int NDIM, typename F>
__device__ __forceinline__ void for_tiles(const Tiles &tl, const unsigned char *tflag, F &&body) {
    for (int t = blockIdx.x; t < tl.nt; t += gridDim.x) {
        const int bx = t % tl.ntx, rr = t / tl.ntx;
        const int by = rr % tl.nty, bz = rr / tl.nty;
        body(bx * 32, by * 8, bz * MW<NDIM>::TZ, tflag ? tflag[t] != 0 : false);
    }
}

// q = A d with d formed on the fly (IT0: d as stored; else d = D^-1 s + beta
// d_prev, written back); alpha = rho / <d, q>.
template <typename T, int NDIM, bool IT0>
__global__ void __launch_bounds__(256) k_pcg_qm(LevelD<T> L, DevScalars *S, double *part, int lev, int it) {
    using W = MW<NDIM>;
    using Z = MZ<NDIM, T>;
    __shared__ T slab[Z::NPL * W::WN];
    const T *dprev = L.d[(it + 1) & 1];
    T *dcur = L.d[it & 1];
    const T beta = IT0 ? T(0) : (T)S->beta[lev];
    const GridD &g = L.g;
    auto op = [&](int q) -> T { return IT0 ? dcur[q] : L.invD[q] * L.s[q] + beta * dprev[q]; };
    T acc[1] = {T(0)};
    const int i = threadIdx.x, j = threadIdx.y;
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int gi = x0 + i, gj = y0 + j;
        const bool in = gi < g.n[0] && gj < g.n[1];
        const int zb = NDIM == 3 ? z0 : 0, zend = NDIM == 3 ? min(z0 + W::TZ, g.n[2]) : 1;
        for (int zs = zb; zs < zend; zs += Z::ZC) {
            __syncthreads();
            load_slab<NDIM, T>(slab, g, x0, y0, zs, op);
            __syncthreads();
            if (!in) continue;
            for (int dz = 0; dz < Z::ZC && zs + dz < zend; ++dz) {
                const int z = zs + dz;
                const T *pc = slab + (NDIM == 3 ? (dz + 1) * W::WN : 0);
                const Nb6<NDIM, T> v = nb6<NDIM>(NDIM == 3 ? pc - W::WN : pc, pc, NDIM == 3 ? pc + W::WN : pc);
                const int idx = gi + g.n[0] * (gj + g.n[1] * z);
                T cp[3], cm[3];
                coefs<T, NDIM>(L, uni, gi, gj, z, idx, cp, cm);
                T Ad = cp[0] * (v.xp - v.c) - cm[0] * (v.c - v.xm) + cp[1] * (v.yp - v.c) - cm[1] * (v.c - v.ym);
                if (NDIM == 3) Ad += cp[2] * (v.zp - v.c) - cm[2] * (v.c - v.zm);
                if (!IT0) dcur[idx] = v.c;
                L.q[idx] = Ad;
                acc[0] += v.c * Ad;
            }
        }
    });
    double out[1];
    if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_Q], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) S->alpha[lev] = out[0] != 0.0 ? S->rho[lev] / out[0] : 0.0;
}

// PCG start after the coarse correction: x = P x_c (injection), s = r - A x,
// d = D^-1 s, rho = <s, d>.
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_pcg_initm(LevelD<T> L, GridD gc, const T *xc, DevScalars *S, double *part,
                                                   int lev) {
    using W = MW<NDIM>;
    using Z = MZ<NDIM, T>;
    __shared__ T slab[Z::NPL * W::WN];
    const GridD &g = L.g;
    const int n0 = g.n[0], n01 = g.n[0] * g.n[1];
    auto op = [&](int q) -> T {
        const int k = q / n01, rem = q - k * n01, j = rem / n0, i = rem - j * n0;
        return xc[(i >> 1) + gc.n[0] * ((j >> 1) + gc.n[1] * (NDIM == 3 ? (k >> 1) : 0))];
    };
    T acc[1] = {T(0)};
    const int i = threadIdx.x, j = threadIdx.y;
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int gi = x0 + i, gj = y0 + j;
        const bool in = gi < g.n[0] && gj < g.n[1];
        const int zb = NDIM == 3 ? z0 : 0, zend = NDIM == 3 ? min(z0 + W::TZ, g.n[2]) : 1;
        for (int zs = zb; zs < zend; zs += Z::ZC) {
            __syncthreads();
            load_slab<NDIM, T>(slab, g, x0, y0, zs, op);
            __syncthreads();
            if (!in) continue;
            for (int dz = 0; dz < Z::ZC && zs + dz < zend; ++dz) {
                const int z = zs + dz;
                const T *pc = slab + (NDIM == 3 ? (dz + 1) * W::WN : 0);
                const Nb6<NDIM, T> v = nb6<NDIM>(NDIM == 3 ? pc - W::WN : pc, pc, NDIM == 3 ? pc + W::WN : pc);
                const int idx = gi + g.n[0] * (gj + g.n[1] * z);
                const T iD = L.invD[idx];
                T sv = T(0);
                if (iD != T(0)) {
                    T cp[3], cm[3];
                    coefs<T, NDIM>(L, uni, gi, gj, z, idx, cp, cm);
                    T Ax = cp[0] * (v.xp - v.c) - cm[0] * (v.c - v.xm) + cp[1] * (v.yp - v.c) - cm[1] * (v.c - v.ym);
                    if (NDIM == 3) Ax += cp[2] * (v.zp - v.c) - cm[2] * (v.c - v.zm);
                    sv = L.r[idx] - Ax;
                }
                const T zz = iD * sv;
                L.x[idx] = v.c;
                L.s[idx] = sv;
                L.d[0][idx] = zz;
                acc[0] += sv * zz;
            }
        }
    });
    double out[1];
    if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_INIT], out))
        if (threadIdx.x == 0 && threadIdx.y == 0) S->rho[lev] = out[0];
}

// Refinement residual r = (b - mean) - A (ph + pl), compensated (exact
// differences, FMA products, two-sum accumulation), at active rows; written to
// the fine level and, when RESTRICT, summed over the 2^n children straight into
// the next level's right-hand side; |r| / |b - mean| -> S->rel.
template <typename T, int NDIM, bool RESTRICT>
__global__ void __launch_bounds__(256) k_residm(LevelD<T> L, const T *b, const T *bl, const T *ph, const T *pl,
                                                LevelD<T> C, DevScalars *S, double *part) {
    using W = MW<NDIM>;
    using Z = MZ<NDIM, T>;
    __shared__ T sh_[Z::NPL * W::WN], sl_[Z::NPL * W::WN];
    __shared__ T rpl[8][33];
    const GridD &g = L.g;
    const T bm = (T)S->bmean;
    const T bml = (T)(S->bmean - (double)bm);
    auto oph = [&](int q) -> T { return ph[q]; };
    auto opl = [&](int q) -> T { return pl[q]; };
    T acc[1] = {T(0)};
    const int i = threadIdx.x, j = threadIdx.y;
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const int gi = x0 + i, gj = y0 + j;
        const bool in = gi < g.n[0] && gj < g.n[1];
        const int zb = NDIM == 3 ? z0 : 0, zend = NDIM == 3 ? min(z0 + W::TZ, g.n[2]) : 1;
        T csum = T(0);  // restriction partial over a z pair
        for (int zs = zb; zs < zend; zs += Z::ZC) {
            __syncthreads();
            load_slab<NDIM, T>(sh_, g, x0, y0, zs, oph);
            load_slab<NDIM, T>(sl_, g, x0, y0, zs, opl);
            __syncthreads();
            for (int dz = 0; dz < Z::ZC && zs + dz < zend; ++dz) {
                const int z = zs + dz;
                T res = T(0);
                if (in) {
                    const int idx = gi + g.n[0] * (gj + g.n[1] * z);
                    if (uni || L.invD[idx] != T(0)) {
                        const T *hc = sh_ + (NDIM == 3 ? (dz + 1) * W::WN : 0);
                        const T *lc = sl_ + (NDIM == 3 ? (dz + 1) * W::WN : 0);
                        const Nb6<NDIM, T> h = nb6<NDIM>(NDIM == 3 ? hc - W::WN : hc, hc, NDIM == 3 ? hc + W::WN : hc);
                        const Nb6<NDIM, T> l = nb6<NDIM>(NDIM == 3 ? lc - W::WN : lc, lc, NDIM == 3 ? lc + W::WN : lc);
                        T cp[3], cm[3];
                        coefs<T, NDIM>(L, uni, gi, gj, z, idx, cp, cm);
                        const T hP[3] = {h.xp, h.yp, h.zp}, hM[3] = {h.xm, h.ym, h.zm};
                        const T lP[3] = {l.xp, l.yp, l.zp}, lM[3] = {l.xm, l.ym, l.zm};
                        T Ah = T(0), Al = T(0);
#pragma unroll
                        for (int a = 0; a < NDIM; ++a) {
                            T th, tl, s, e;
                            if (cp[a] == cm[a]) {
                                // equal faces: c [(p+ - p) - (p - p-)] formed exactly
                                T hp, ehp, hm, ehm, s2, es;
                                two_sum(hP[a], -h.c, hp, ehp);
                                two_sum(h.c, -hM[a], hm, ehm);
                                two_sum(hp, -hm, s2, es);
                                const T lo = ((ehp - ehm) + es) + ((lP[a] - l.c) - (l.c - lM[a]));
                                th = cm[a] * s2;
                                tl = fma(cm[a], s2, -th) + cm[a] * lo;
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                            } else {
                                face_term(hP[a], lP[a], h.c, l.c, cp[a], th, tl);
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                                face_term(hM[a], lM[a], h.c, l.c, cm[a], th, tl);
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                            }
                        }
                        T r1, e1, r2, e2;
                        two_sum(b[idx], -bm, r1, e1);
                        two_sum(r1, -Ah, r2, e2);
                        res = r2 + (((e1 + e2) + (bl[idx] - bml)) - Al);
                        acc[0] += res * res;
                    }
                    L.r[idx] = res;
                }
                if (RESTRICT) {
                    // children (2i..2i+1, 2j..2j+1, 2k..2k+1): x pairs by shuffle,
                    // y pairs through shared memory, z pairs in a register
                    const T v = res + __shfl_xor_sync(0xffffffffu, res, 1);
                    rpl[j][i] = v;
                    __syncthreads();
                    if ((i & 1) == 0 && (j & 1) == 0) {
                        csum += v + rpl[j + 1][i];
                        if (NDIM == 2 || (z & 1) == 1) {
                            const int ci = gi >> 1, cj = gj >> 1, ck = NDIM == 3 ? (z >> 1) : 0;
                            if (ci < C.g.n[0] && cj < C.g.n[1]) C.r[ci + C.g.n[0] * (cj + C.g.n[1] * ck)] = csum;
                            csum = T(0);
                        }
                    }
                    __syncthreads();
                }
            }
        }
    });
    double out[1];
    if (grid_reduce<1, false, T>(acc, part, &S->counters[RS_RESID], out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            S->rnorm2 = out[0];
            const double bn = S->bnorm;
            const double rel = bn > 0 ? sqrt(out[0]) / bn : (out[0] > 0 ? 1e300 : 0.0);
            S->rel = rel;
            if (!(rel == rel) || !(bn == bn) || rel >= 1e300) S->status |= 1;
        }
    }
}
