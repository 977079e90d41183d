// k_resid.cuh -- refinement residual of the projection's Poisson solve, with
// the restriction to the next level fused.
//
// The solve iterates on p = ph + pl (a float pair) and needs r = b - A p with
// an error well below the FP32 rounding of A p itself (Sec. 2 operator; the
// V-cycle of Sec. 4.2 reduces r, the pair carries the correction). The
// column-marching layout is that of the smoother kernels.
#pragma once
#include "k_mg_march.cuh"

// Refinement residual r = (b - mean) - A (ph + pl), compensated (exact
// differences, FMA products, two-sum accumulation), at active rows; written to
// the fine level and, when RESTRICT, summed over the 2^n children straight into
// the next level's right-hand side; |r| / |b - mean| -> S->rel. A column is
// processed in batches of HB planes whose loads are all issued first.
template <typename T, int NDIM, bool RESTRICT>
__global__ void __launch_bounds__(256) k_residm(LevelD<T> L, const T *__restrict__ b, const T *__restrict__ bl,
                                                const T *__restrict__ ph, const T *__restrict__ pl, LevelD<T> C,
                                                DevScalars *S, double *part) {
    constexpr int TZ = MT<NDIM>::TZ;
    constexpr int HB = 1;
    __shared__ T rpl[2][8][33];   // double-buffered by plane parity (3D)
    const GridD &g = L.g;
    const T bm = (T)S->bmean;
    const T bml = (T)(S->bmean - (double)bm);
    const int plane = g.n[0] * g.n[1];
    const bool pz = g.per[2] != 0;
    T *__restrict__ rout = L.r;
    T acc[1] = {T(0)};
    for_tiles<NDIM>(L.tl, L.tflag, [&](int x0, int y0, int z0, bool uni) {
        const Col c = column(g, x0, y0);
        const int base = (c.in ? c.i : 0) + g.n[0] * (c.in ? c.j : 0);
        const int zb = NDIM == 3 ? z0 : 0, nz = NDIM == 3 ? min(TZ, g.n[2] - z0) : 1;
        // uniform tile away from every non-periodic domain face
        const bool plain = uni && (g.per[0] || (x0 > 0 && x0 + 32 < g.n[0])) &&
                           (g.per[1] || (y0 > 0 && y0 + 8 < g.n[1])) &&
                           (NDIM == 2 || pz || (zb > 0 && zb + nz < g.n[2]));
        T csum = T(0);
        for (int hb = 0; hb < nz; hb += HB) {
            // batch loads: z column (HB + 2), x/y neighbours, b pair
            T hz[HB + 2], lz[HB + 2], hx[4][HB], lx[4][HB], bv[HB], blv[HB];
#pragma unroll
            for (int t = 0; t < HB + 2; ++t) {
                hz[t] = lz[t] = T(0);
                if (c.in && (NDIM == 3 ? hb + t <= nz + 1 - 0 && hb + t - 1 <= nz : t == 1)) {
                    const int q = NDIM == 3 ? base + plane * edge_idx(zb + hb - 1 + t, g.n[2], pz) : base;
                    hz[t] = ph[q];
                    lz[t] = pl[q];
                }
            }
#pragma unroll
            for (int t = 0; t < HB; ++t)
                if (c.in && hb + t < nz) {
                    const int idx = base + plane * (zb + hb + t);
                    const int off[4] = {c.oxm, c.oxp, c.oym, c.oyp};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        hx[u][t] = ph[idx + off[u]];
                        lx[u][t] = pl[idx + off[u]];
                    }
                    bv[t] = b[idx];
                    blv[t] = bl[idx];
                }
#pragma unroll
            for (int t = 0; t < HB; ++t) {
                const int k = zb + hb + t;
                const bool live = hb + t < nz;
                const int idx = base + plane * k;
                T res = T(0);
                if (c.in && live) {
                    if (uni || L.invD[idx] != T(0)) {
                        const T hc = hz[t + 1], lc = lz[t + 1];
                        const T hP[3] = {hx[1][t], hx[3][t], hz[t + 2]}, hM[3] = {hx[0][t], hx[2][t], hz[t]};
                        const T lP[3] = {lx[1][t], lx[3][t], lz[t + 2]}, lM[3] = {lx[0][t], lx[2][t], lz[t]};
                        T Ah = T(0), Al = T(0);
                        if (plain) {
                            // every face carries cu (a power of two: exact
                            // scaling): A p = cu sum_a [(p+ - p) - (p - p-)], the
                            // second differences formed and summed exactly
#pragma unroll
                            for (int a = 0; a < NDIM; ++a) {
                                T d1, e1, d2, e2, s2, es, s, e;
                                two_sum(hP[a], -hc, d1, e1);
                                two_sum(hc, -hM[a], d2, e2);
                                two_sum(d1, -d2, s2, es);
                                two_sum(Ah, s2, s, e);
                                Ah = s;
                                Al += e + (((e1 - e2) + es) + ((lP[a] - lc) - (lc - lM[a])));
                            }
                            Ah *= L.cu;
                            Al *= L.cu;
                        } else {
                        T cp[3], cm[3];
                        coefs<T, NDIM>(L, uni, c.i, c.j, k, idx, cp, cm);
#pragma unroll
                        for (int a = 0; a < NDIM; ++a) {
                            T th, tl, s, e;
                            if (cp[a] == cm[a]) {
                                // equal faces: c [(p+ - p) - (p - p-)] formed exactly
                                T d1, e1, d2, e2, s2, es;
                                two_sum(hP[a], -hc, d1, e1);
                                two_sum(hc, -hM[a], d2, e2);
                                two_sum(d1, -d2, s2, es);
                                const T lo = ((e1 - e2) + es) + ((lP[a] - lc) - (lc - lM[a]));
                                th = cm[a] * s2;
                                tl = fma(cm[a], s2, -th) + cm[a] * lo;
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                            } else {
                                face_term(hP[a], lP[a], hc, lc, cp[a], th, tl);
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                                face_term(hM[a], lM[a], hc, lc, cm[a], th, tl);
                                two_sum(Ah, th, s, e);
                                Ah = s;
                                Al += e + tl;
                            }
                        }
                        }
                        T r1, e1, r2, e2;
                        two_sum(bv[t], -bm, r1, e1);
                        two_sum(r1, -Ah, r2, e2);
                        res = r2 + (((e1 + e2) + (blv[t] - bml)) - Al);
                        acc[0] += res * res;
                    }
                    rout[idx] = res;
                }
                if (RESTRICT && live) {
                    // children (2i..2i+1, 2j..2j+1, 2k..2k+1): x pairs by shuffle,
                    // y pairs through shared memory, z pairs in a register
                    const int i = threadIdx.x, j = threadIdx.y;
                    const int pb = NDIM == 3 ? (k & 1) : 0;
                    const T v = res + __shfl_xor_sync(0xffffffffu, res, 1);
                    rpl[pb][j][i] = v;
                    __syncthreads();
                    if ((i & 1) == 0 && (j & 1) == 0) {
                        csum += v + rpl[pb][j + 1][i];
                        if (NDIM == 2 || (k & 1) == 1) {
                            const int ci = c.i >> 1, cj = c.j >> 1, ck = NDIM == 3 ? (k >> 1) : 0;
                            if (ci < C.g.n[0] && cj < C.g.n[1]) C.r[ci + C.g.n[0] * (cj + C.g.n[1] * ck)] = csum;
                            csum = T(0);
                        }
                    }
                    // (3D: the next plane writes the other buffer, and the one
                    // after it is written only past the next plane's barrier)
                    if (NDIM == 2) __syncthreads();
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
