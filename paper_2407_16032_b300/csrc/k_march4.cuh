// k_march4.cuh -- plane-marching smoother stencils of FP32 3D levels.
//
// The operator is the variable-coefficient Poisson operator of the projection
// (Sec. 2; the PCG smoother of the multigrid, Sec. 4.2):
//   (A p)[I] = sum_a c_a[I+e_a](p[I+e_a]-p[I]) - c_a[I](p[I]-p[I-e_a]).
// A block of 256 threads owns a 128 x 8 tile of the (x, y) plane and marches
// it through KZ planes along z. Each thread owns 4 consecutive x cells of one
// row (16-byte loads and stores). The operand of the stencil is formed plane
// by plane into a ring of three shared planes (the tile with a one-cell ring
// in x and y); the thread keeps its own column's three planes in registers
// (the z neighbours), takes the x neighbours of its 4 cells from its own
// registers and, across lanes, by warp shuffles, and the y neighbours from
// the shared plane. One barrier per plane. The loads of plane k + 2 are in
// flight while plane k's operator is applied.
//
// Per-cell arithmetic is the same as the column kernels' (k_mg_march.cuh):
// uniform tiles away from non-periodic domain faces take A = cu (sum of the six
// neighbours - 6 p); other cells take their coefficients from the position
// (uniform tiles) or from the coefficient arrays.
#pragma once
#include "k_mg_march.cuh"

#include <type_traits>

namespace m4 {
constexpr int TX = 128, TY = 8;   // in-plane tile: 32 lanes x 4 cells, 8 warps
#ifndef M4_KZ
#define M4_KZ 16
#endif
constexpr int KZ = M4_KZ;         // planes marched per tile
constexpr int PADX = 4;           // shared row: PADX | TX cells | PADX (16-byte aligned)
constexpr int RW = TX + 2 * PADX;

// Flag of the 32 x 8 x 8 tile of cell (i, j, k) (the tiles of LevelD::tl).
__device__ __forceinline__ bool tile_uniform(const LevelD<float> &L, int i, int j, int k) {
    return L.tflag[(i >> 5) + L.tl.ntx * ((j >> 3) + L.tl.nty * (k >> 3))] != 0;
}

// The 32 x 8 x 8 tile of (i, j, k) is uniform and away from every
// non-periodic domain face: all of its cells have 2n faces of coefficient cu.
__device__ __forceinline__ bool tile_plain(const LevelD<float> &L, int i, int j, int k) {
    const GridD &g = L.g;
    const int x0 = i & ~31, y0 = j & ~7, z0 = k & ~7;
    return tile_uniform(L, i, j, k) && (g.per[0] || (x0 > 0 && x0 + 32 < g.n[0])) &&
           (g.per[1] || (y0 > 0 && y0 + 8 < g.n[1])) && (g.per[2] || (z0 > 0 && z0 + 8 < g.n[2]));
}

// 1/D of cell (i, j, k): from the position in a uniform tile (all faces cu
// except non-periodic domain faces), else from the array.
__device__ __forceinline__ float invd_cell(const LevelD<float> &L, const float *idtab, int i, int j, int k, int idx) {
    if (!tile_uniform(L, i, j, k)) return L.invD[idx];
    const GridD &g = L.g;
    int nf = 6;
    if (!g.per[0]) nf -= (i == 0) + (i == g.n[0] - 1);
    if (!g.per[1]) nf -= (j == 0) + (j == g.n[1] - 1);
    if (!g.per[2]) nf -= (k == 0) + (k == g.n[2] - 1);
    return idtab[nf];
}

__device__ __forceinline__ float f4get(const float4 &v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// A d at the 4 cells (i..i+3, j, k) of a thread: dc centre, xm / xp the x
// neighbours of cells 0 and 3, ym / yp the rows y -/+ 1, zm / zp the planes.
__device__ __forceinline__ float4 apply4(const LevelD<float> &L, bool plain, bool uni, int i, int j, int k, int idx,
                                         const float4 &dc, float xm, float xp, const float4 &ym, const float4 &yp,
                                         const float4 &zm, const float4 &zp) {
    const float c[4] = {dc.x, dc.y, dc.z, dc.w};
    const float l[4] = {xm, dc.x, dc.y, dc.z}, r[4] = {dc.y, dc.z, dc.w, xp};
    float out[4];
    if (plain) {
        const float cu = L.cu;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float nb = (r[e] + l[e]) + (f4get(yp, e) + f4get(ym, e));
            nb += f4get(zp, e) + f4get(zm, e);
            out[e] = cu * (nb - 6.f * c[e]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float cp[3], cm[3];
            coefs<float, 3>(L, uni, i + e, j, k, idx + e, cp, cm);
            float Ad = cp[0] * (r[e] - c[e]) - cm[0] * (c[e] - l[e]) + cp[1] * (f4get(yp, e) - c[e]) -
                       cm[1] * (c[e] - f4get(ym, e));
            Ad += cp[2] * (f4get(zp, e) - c[e]) - cm[2] * (c[e] - f4get(zm, e));
            out[e] = Ad;
        }
    }
    return make_float4(out[0], out[1], out[2], out[3]);
}
}  // namespace m4

// Per-thread asynchronous copies (cp.async) of global data into shared memory:
// 16 bytes (both addresses 16-byte aligned) or 4 bytes. A thread's copies are
// grouped per plane (commit) and waited for by count (wait_group): each thread
// waits only for its own copies, and only reads the cells it copied itself
// until the next block barrier.
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Search direction and operator in one pass (PCG iteration, first half):
//   d = D^-1 s + beta d_old  (d = D^-1 s on the first iteration),
//   q = A d,   alpha = rho / <d, q>.
// d_old and d are different buffers. Requires n[0] % 4 == 0. The planes of s
// (and d_old) stream through M4_STAGES shared stages: each thread copies its
// own cells of plane k + M4_STAGES - 2 while plane k is worked on, forms d in
// place in the stage, and after one block barrier the stage is the stencil
// plane of the operator. Everything that does not change along the march (the
// uniform flags of the 32 x 8 x 8 tiles, the domain faces of the thread's
// cells, its addresses) is set up once per tile.
#ifndef M4_STAGES
#define M4_STAGES 5
#endif
#ifndef M4_MINB
#define M4_MINB 3
#endif
template <bool FIRST>
constexpr size_t pcg_dq4_smem() {
    return (size_t)M4_STAGES * (FIRST ? 1 : 2) * (m4::TY + 2) * m4::RW * sizeof(float);
}

namespace m4 {
// 1/D of a uniform cell with `nb` non-periodic domain faces: idtab[6 - nb].
// Domain faces of a cell: lower x face at i == 0, upper at i == n0 - 1, etc.
__device__ __forceinline__ int xfaces(const GridD &g, int i) {
    return g.per[0] ? 0 : (i == 0) + (i == g.n[0] - 1);
}
__device__ __forceinline__ int yfaces(const GridD &g, int j) {
    return g.per[1] ? 0 : (j == 0) + (j == g.n[1] - 1);
}
__device__ __forceinline__ int zfaces(const GridD &g, int k) {
    return g.per[2] ? 0 : (k == 0) + (k == g.n[2] - 1);
}
}  // namespace m4

template <bool FIRST>
__global__ void __launch_bounds__(256, M4_MINB) k_pcg_dq4(LevelD<float> L, const float *__restrict__ dold,
                                                    float *__restrict__ dnew, DevScalars *S, double *part, int lev) {
    using namespace m4;
    constexpr int P = M4_STAGES, NA = FIRST ? 1 : 2;
    constexpr int SW = NA * (TY + 2) * RW;   // floats per stage
    constexpr int AW = (TY + 2) * RW;        // floats per array within a stage
    extern __shared__ __align__(16) float smem4[];
    __shared__ float idtab[8];
    const GridD &g = L.g;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], plane = n0 * n1;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float beta = FIRST ? 0.f : (float)S->beta[lev];
    const float cu = L.cu;
    const float *__restrict__ s_g = L.s;
    const float *__restrict__ iD_g = L.invD;
    float *__restrict__ q = L.q;
    if (threadIdx.x < 8) idtab[threadIdx.x] = threadIdx.x > 0 ? -1.f / (float(threadIdx.x) * cu) : 0.f;
    __syncthreads();
    const float idc = idtab[6];
    const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY, ntz = (n2 + KZ - 1) / KZ;
    float acc[1] = {0.f};
    for (int t = blockIdx.x; t < ntx * nty * ntz; t += gridDim.x) {
        const int bx = t % ntx, rr = t / ntx, by = rr % nty, bz = rr / nty;
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * KZ;
        const int nx = min(TX, n0 - x0), ny = min(TY, n1 - y0), z1 = min(z0 + KZ, n2);
        const int i = x0 + 4 * lane, j = y0 + w;
        const bool in = 4 * lane < nx && w < ny;
        const int last = nx / 4 - 1;
        // ring cells copied and formed by this thread: row 0 (warps 0-3) or
        // ny + 1 (warps 4-7), 32 cells each; lane 0 / 1 the left / right ring
        // cell of row w
        const int hc = 32 * (w & 3) + lane;
        const bool hin = hc < nx;
        const int hx = x0 + hc;
        const int hj = w < 4 ? edge_idx(y0 - 1, n1, py) : edge_idx(y0 + ny, n1, py);
        const int hrow = w < 4 ? 0 : ny + 1;
        const bool xin = w < ny && lane < 2;
        const int xi = lane == 0 ? edge_idx(x0 - 1, n0, px) : edge_idx(x0 + nx, n0, px);
        const int xcol = lane == 0 ? PADX - 1 : PADX + nx;
        const int np = z1 - z0 + 2;   // planes z0-1 .. z1 (relative index r = 0 .. np-1)
        const int klo = edge_idx(z0 - 1, n2, pz), khi = edge_idx(z1, n2, pz);
        // uniform flags of the z-slots of the march: 0 = plane z0-1, 1 = planes
        // z0..z0+7, 2 = z0+8..z0+15, 3 = plane z1 (bit 0 own cells, 1 ring row
        // cell, 2 ring column cell)
        unsigned uflag = 0;
        bool all_uni = true;
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            const int kr = sl == 0 ? klo : (sl == 3 ? khi : min(z0 + 8 * (sl - 1), n2 - 1));
            unsigned f = 0;
            if (in && tile_uniform(L, i, j, kr)) f |= 1;
            if (hin && tile_uniform(L, hx, hj, kr)) f |= 2;
            if (xin && tile_uniform(L, xi, j, kr)) f |= 4;
            const unsigned need = (in ? 1u : 0u) | (hin ? 2u : 0u) | (xin ? 4u : 0u);
            if ((f & need) != need) all_uni = false;
            uflag |= f << (3 * sl);
        }
        // one path for the whole tile: every cell and ring cell uniform, or not
        all_uni = __syncthreads_and(all_uni);
        // domain faces (x, y) of the thread's cells and ring cells
        const int fy = yfaces(g, j);
        const int fx0 = xfaces(g, i), fx3 = xfaces(g, i + 3);
        const bool edge = fx0 != 0 || fx3 != 0 || fy != 0;   // some own face lies on the domain boundary
        const bool bxl = !px && i == 0, bxr = !px && i + 3 == n0 - 1;   // domain x faces of cells 0 and 3
        const bool byl = !py && j == 0, byr = !py && j == n1 - 1;        // domain y faces of the row
        const int fh = xfaces(g, hx) + yfaces(g, hj);
        const int fxr = xfaces(g, xi) + yfaces(g, j);
        // 32-bit element offsets of the thread's cells in plane 0
        const int oown = i + n0 * j, oh = hx + n0 * hj, ox = xi + n0 * j;
        auto kof = [&](int r) { return r == 0 ? klo : (r == np - 1 ? khi : z0 - 1 + r); };
        auto slot = [&](int r) { return r == 0 ? 0 : (r == np - 1 ? 3 : 1 + ((r - 1) >> 3)); };
        auto stage_ptr = [&](int st) { return smem4 + st * SW; };
        // copy this thread's cells of relative plane r into stage st (nothing if r >= np); one group
        auto issue = [&](int r, int st) {
            if (r < np) {
                const int pb = plane * kof(r);
                float *sa = stage_ptr(st);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float *gsrc = (a == 0 ? s_g : dold) + pb;
                    if (in) cpa16(sa + (w + 1) * RW + PADX + 4 * lane, gsrc + oown);
                    if (hin) cpa4(sa + hrow * RW + PADX + hc, gsrc + oh);
                    if (xin) cpa4(sa + (w + 1) * RW + xcol, gsrc + ox);
                    sa += AW;
                }
            }
            cpa_commit();
        };
        // the march, specialised at compile time for uniform tiles (UNI: 1/D
        // and the coefficients from the position) or general ones
        auto march = [&](auto uni_tag) {
            constexpr bool UNI = decltype(uni_tag)::value;
            // form d in place for this thread's cells of relative plane r (its
            // copies have landed); returns its own 4 values
            auto form = [&](int r, int st) -> float4 {
                float *sa = stage_ptr(st);
                const int kk = kof(r);
                const int fz = zfaces(g, kk);
                const unsigned f = UNI ? 7u : uflag >> (3 * slot(r));
                float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in) {
                    float iv[4];
                    if (f & 1) {
                        if (!edge && fz == 0) {
                            iv[0] = iv[1] = iv[2] = iv[3] = idc;
                        } else {
                            const int b = fy + fz;
                            iv[0] = idtab[6 - b - fx0];
                            iv[1] = iv[2] = idtab[6 - b];
                            iv[3] = idtab[6 - b - fx3];
                        }
                    } else {
                        const float4 v = *(const float4 *)(iD_g + plane * kk + oown);
                        iv[0] = v.x; iv[1] = v.y; iv[2] = v.z; iv[3] = v.w;
                    }
                    float4 *sp = (float4 *)(sa + (w + 1) * RW + PADX + 4 * lane);
                    const float4 sv = *sp;
                    if (FIRST) {
                        dv = make_float4(iv[0] * sv.x, iv[1] * sv.y, iv[2] * sv.z, iv[3] * sv.w);
                    } else {
                        const float4 dd = *(const float4 *)(sa + AW + (w + 1) * RW + PADX + 4 * lane);
                        dv = make_float4(iv[0] * sv.x + beta * dd.x, iv[1] * sv.y + beta * dd.y,
                                         iv[2] * sv.z + beta * dd.z, iv[3] * sv.w + beta * dd.w);
                    }
                    *sp = dv;
                }
                if (hin) {
                    float *c = sa + hrow * RW + PADX + hc;
                    const float iv = (f & 2) ? idtab[6 - fh - fz] : iD_g[plane * kk + oh];
                    *c = FIRST ? iv * *c : iv * *c + beta * c[AW];
                }
                if (xin) {
                    float *c = sa + (w + 1) * RW + xcol;
                    const float iv = (f & 4) ? idtab[6 - fxr - fz] : iD_g[plane * kk + ox];
                    *c = FIRST ? iv * *c : iv * *c + beta * c[AW];
                }
                return dv;
            };
#pragma unroll
            for (int r = 0; r < P; ++r) issue(r, r);
            cpa_wait<P - 1>();
            float4 dm = form(0, 0);
            cpa_wait<P - 2>();
            float4 dcv = form(1, 1);
            int sti = 2;   // stage of relative plane r + 1 in the loop below
            int stc = 1;   // stage of the centre plane
            int stf = 0;   // stage to refill after the barrier (plane r - 1)
            for (int k = z0; k < z1; ++k) {
                const int r = k - z0 + 1;   // relative plane of k
                cpa_wait<P - 3>();
                const float4 dp = form(r + 1, sti);
                __syncthreads();
                // every read of plane k - 1's stage is done: refill it with plane r - 1 + P
                issue(r - 1 + P, stf);
                const float *sc = stage_ptr(stc);
                float xm = __shfl_up_sync(0xffffffffu, dcv.w, 1);
                float xp = __shfl_down_sync(0xffffffffu, dcv.x, 1);
                if (in) {
                    if (lane == 0) xm = sc[(w + 1) * RW + PADX - 1];
                    if (lane == last) xp = sc[(w + 1) * RW + PADX + nx];
                    const float4 ym = *(const float4 *)(sc + w * RW + PADX + 4 * lane);
                    const float4 yp = *(const float4 *)(sc + (w + 2) * RW + PADX + 4 * lane);
                    const int id = plane * k + oown;
                    const bool uni = UNI || ((uflag >> (3 * slot(r))) & 1);
                    float4 Ad;
                    if (uni) {
                        // a neighbour across a non-periodic domain face takes the
                        // centre value: that face's term is exactly zero
                        if (bxl) xm = dcv.x;
                        if (bxr) xp = dcv.w;
                        const float4 zm = (!pz && k == 0) ? dcv : dm, zp = (!pz && k == n2 - 1) ? dcv : dp;
                        Ad = apply4(L, true, true, i, j, k, id, dcv, xm, xp, byl ? dcv : ym, byr ? dcv : yp, zm, zp);
                    } else {
                        Ad = apply4(L, false, false, i, j, k, id, dcv, xm, xp, ym, yp, dm, dp);
                    }
                    *(float4 *)(dnew + id) = dcv;
                    *(float4 *)(q + id) = Ad;
                    acc[0] += dcv.x * Ad.x;
                    acc[0] += dcv.y * Ad.y;
                    acc[0] += dcv.z * Ad.z;
                    acc[0] += dcv.w * Ad.w;
                }
                dm = dcv;
                dcv = dp;
                stf = stc;
                stc = sti;
                sti = sti + 1 == P ? 0 : sti + 1;
            }
        };
        if (all_uni) march(std::true_type{});
        else march(std::false_type{});
        cpa_wait<0>();
        __syncthreads();   // every read of the stages is done before the next tile's copies
    }
    double out[1];
    if (grid_reduce<1, false, float>(acc, part, &S->counters[RS_Q], out))
        if (threadIdx.x == 0) S->alpha[lev] = out[0] != 0.0 ? S->rho[lev] / out[0] : 0.0;
}

// ---------------------------------------------------------------- residual
// Refinement residual r = (b - mean) - A (ph + pl) of the fine level, with the
// per-cell compensated arithmetic of k_residm (exact differences, two-sum
// accumulation; the same operations in the same order), on the plane march:
// the pair (ph, pl) streams through the stages with its ring, b and bl are
// loaded a plane ahead. When RESTRICT, the 2 x 2 x 2 children sums go to the
// next level's right-hand side: x pairs within a thread, y pairs between the
// warps of rows 2m and 2m + 1 through shared memory (behind the next plane's
// barrier), z pairs in a register. |r| / |b - mean| -> S->rel.
template <bool RESTRICT>
constexpr size_t resid4_smem() {
    return (size_t)M4_STAGES * 2 * (m4::TY + 2) * m4::RW * sizeof(float);
}

namespace m4 {
// residual of one cell from its centre pair and the six neighbour pairs, as k_residm
__device__ __forceinline__ float resid_cell(const LevelD<float> &L, bool plain, bool uni, int i, int j, int k, int idx,
                                            float hc, float lc, const float (&hP)[3], const float (&lP)[3],
                                            const float (&hM)[3], const float (&lM)[3], float bv, float blv, float bm,
                                            float bml) {
    float Ah = 0.f, Al = 0.f;
    if (plain) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float d1, e1, d2, e2, s2, es, s, e;
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
        float cp[3], cm[3];
        coefs<float, 3>(L, uni, i, j, k, idx, cp, cm);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float th, tl, s, e;
            if (cp[a] == cm[a]) {
                float d1, e1, d2, e2, s2, es;
                two_sum(hP[a], -hc, d1, e1);
                two_sum(hc, -hM[a], d2, e2);
                two_sum(d1, -d2, s2, es);
                const float lo = ((e1 - e2) + es) + ((lP[a] - lc) - (lc - lM[a]));
                th = cm[a] * s2;
                tl = fmaf(cm[a], s2, -th) + cm[a] * lo;
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
    float r1, e1, r2, e2;
    two_sum(bv, -bm, r1, e1);
    two_sum(r1, -Ah, r2, e2);
    return r2 + (((e1 + e2) + (blv - bml)) - Al);
}
}  // namespace m4

template <bool RESTRICT>
__global__ void __launch_bounds__(256, 2) k_resid4(LevelD<float> L, const float *__restrict__ b,
                                                   const float *__restrict__ bl, const float *__restrict__ ph,
                                                   const float *__restrict__ pl, LevelD<float> C, DevScalars *S,
                                                   double *part) {
    using namespace m4;
    constexpr int P = M4_STAGES;
    constexpr int AW = (TY + 2) * RW, SW = 2 * AW;
    extern __shared__ __align__(16) float smem4[];
    __shared__ __align__(8) float rbuf[2][4][64];   // x-pair sums of the odd rows, by plane parity
    const GridD &g = L.g;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], plane = n0 * n1;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float bm = (float)S->bmean;
    const float bml = (float)(S->bmean - (double)bm);
    float *__restrict__ rout = L.r;
    const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY, ntz = (n2 + KZ - 1) / KZ;
    float acc[1] = {0.f};
    for (int t = blockIdx.x; t < ntx * nty * ntz; t += gridDim.x) {
        const int bx = t % ntx, rr = t / ntx, by = rr % nty, bz = rr / nty;
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * KZ;
        const int nx = min(TX, n0 - x0), ny = min(TY, n1 - y0), z1 = min(z0 + KZ, n2);
        const int i = x0 + 4 * lane, j = y0 + w;
        const bool in = 4 * lane < nx && w < ny;
        const int last = nx / 4 - 1;
        const int hc = 32 * (w & 3) + lane;
        const bool hin = hc < nx;
        const int hx = x0 + hc;
        const int hj = w < 4 ? edge_idx(y0 - 1, n1, py) : edge_idx(y0 + ny, n1, py);
        const int hrow = w < 4 ? 0 : ny + 1;
        const bool xin = w < ny && lane < 2;
        const int xi = lane == 0 ? edge_idx(x0 - 1, n0, px) : edge_idx(x0 + nx, n0, px);
        const int xcol = lane == 0 ? PADX - 1 : PADX + nx;
        const int np = z1 - z0 + 2;
        const int klo = edge_idx(z0 - 1, n2, pz), khi = edge_idx(z1, n2, pz);
        // the whole tile is uniform (its cells' faces and their neighbours'):
        // the flags of the tiles its cells lie in (the ring needs no flag: the
        // operand is the pressure itself)
        bool all_uni = true;
        unsigned uflag = 0;
#pragma unroll
        for (int sl = 1; sl < 3; ++sl) {
            const int kr = min(z0 + 8 * (sl - 1), n2 - 1);
            const bool u = !in || tile_uniform(L, i, j, kr);
            if (!u) all_uni = false;
            uflag |= (u ? 1u : 0u) << sl;
        }
        all_uni = __syncthreads_and(all_uni);
        const bool bxl = !px && i == 0, bxr = !px && i + 3 == n0 - 1;   // domain x faces of cells 0 and 3
        const bool byl = !py && j == 0, byr = !py && j == n1 - 1;        // domain y faces of the row
        const int oown = i + n0 * j, oh = hx + n0 * hj, ox = xi + n0 * j;
        auto kof = [&](int r) { return r == 0 ? klo : (r == np - 1 ? khi : z0 - 1 + r); };
        auto stage_ptr = [&](int st) { return smem4 + st * SW; };
        auto issue = [&](int r, int st) {
            if (r < np) {
                const int pb = plane * kof(r);
                float *sa = stage_ptr(st);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float *gsrc = (a == 0 ? ph : pl) + pb;
                    if (in) cpa16(sa + (w + 1) * RW + PADX + 4 * lane, gsrc + oown);
                    if (hin) cpa4(sa + hrow * RW + PADX + hc, gsrc + oh);
                    if (xin) cpa4(sa + (w + 1) * RW + xcol, gsrc + ox);
                    sa += AW;
                }
            }
            cpa_commit();
        };
        auto own = [&](int st, float4 &h, float4 &l) {
            const float *sa = stage_ptr(st) + (w + 1) * RW + PADX + 4 * lane;
            h = *(const float4 *)sa;
            l = *(const float4 *)(sa + AW);
        };
        auto march = [&](auto uni_tag) {
            constexpr bool UNI = decltype(uni_tag)::value;
#pragma unroll
            for (int r = 0; r < P; ++r) issue(r, r);
            float4 hm, lm, hcv, lcv, hp, lp, bv, blv;
            cpa_wait<P - 1>();
            own(0, hm, lm);
            cpa_wait<P - 2>();
            own(1, hcv, lcv);
            if (in) {
                bv = *(const float4 *)(b + plane * z0 + oown);
                blv = *(const float4 *)(bl + plane * z0 + oown);
            }
            float cs0 = 0.f, cs1 = 0.f;   // z-pair sums of the coarse cells (even rows)
            int sti = 2, stc = 1, stf = 0;
            for (int k = z0; k < z1; ++k) {
                const int r = k - z0 + 1;
                cpa_wait<P - 3>();
                own(sti, hp, lp);
                __syncthreads();
                issue(r - 1 + P, stf);
                // b of the next plane in flight during this one
                float4 bn = bv, bln = blv;
                if (in && k + 1 < z1) {
                    bn = *(const float4 *)(b + plane * (k + 1) + oown);
                    bln = *(const float4 *)(bl + plane * (k + 1) + oown);
                }
                const float *sc = stage_ptr(stc);
                const float4 ym_h = *(const float4 *)(sc + w * RW + PADX + 4 * lane);
                const float4 yp_h = *(const float4 *)(sc + (w + 2) * RW + PADX + 4 * lane);
                const float4 ym_l = *(const float4 *)(sc + AW + w * RW + PADX + 4 * lane);
                const float4 yp_l = *(const float4 *)(sc + AW + (w + 2) * RW + PADX + 4 * lane);
                float xmh = __shfl_up_sync(0xffffffffu, hcv.w, 1), xml = __shfl_up_sync(0xffffffffu, lcv.w, 1);
                float xph = __shfl_down_sync(0xffffffffu, hcv.x, 1), xpl = __shfl_down_sync(0xffffffffu, lcv.x, 1);
                float res[4] = {0.f, 0.f, 0.f, 0.f};
                if (in) {
                    if (lane == 0) { xmh = sc[(w + 1) * RW + PADX - 1]; xml = sc[AW + (w + 1) * RW + PADX - 1]; }
                    if (lane == last) { xph = sc[(w + 1) * RW + PADX + nx]; xpl = sc[AW + (w + 1) * RW + PADX + nx]; }
                    const int id = plane * k + oown;
                    const bool uni = UNI || ((uflag >> (1 + ((k - z0) >> 3))) & 1);
                    // in uniform tiles a neighbour across a non-periodic domain
                    // face takes the centre pair: that face's term is exactly zero
                    float4 yph = yp_h, ypl = yp_l, ymh = ym_h, yml = ym_l, zph = hp, zpl = lp, zmh = hm, zml = lm;
                    if (uni) {
                        if (bxl) { xmh = hcv.x; xml = lcv.x; }
                        if (bxr) { xph = hcv.w; xpl = lcv.w; }
                        if (byl) { ymh = hcv; yml = lcv; }
                        if (byr) { yph = hcv; ypl = lcv; }
                        if (!pz && k == 0) { zmh = hcv; zml = lcv; }
                        if (!pz && k == n2 - 1) { zph = hcv; zpl = lcv; }
                    }
                    const bool plain = uni;
                    const float ch[4] = {hcv.x, hcv.y, hcv.z, hcv.w}, cl[4] = {lcv.x, lcv.y, lcv.z, lcv.w};
                    const float lh[4] = {xmh, hcv.x, hcv.y, hcv.z}, ll[4] = {xml, lcv.x, lcv.y, lcv.z};
                    const float rh[4] = {hcv.y, hcv.z, hcv.w, xph}, rl[4] = {lcv.y, lcv.z, lcv.w, xpl};
                    const float bb[4] = {bv.x, bv.y, bv.z, bv.w}, bb2[4] = {blv.x, blv.y, blv.z, blv.w};
                    float ivs[4] = {-1.f, -1.f, -1.f, -1.f};
                    if (!uni) {
                        const float4 v = *(const float4 *)(L.invD + id);
                        ivs[0] = v.x; ivs[1] = v.y; ivs[2] = v.z; ivs[3] = v.w;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (ivs[e] != 0.f) {
                            const float hP[3] = {rh[e], f4get(yph, e), f4get(zph, e)};
                            const float lP[3] = {rl[e], f4get(ypl, e), f4get(zpl, e)};
                            const float hM[3] = {lh[e], f4get(ymh, e), f4get(zmh, e)};
                            const float lM[3] = {ll[e], f4get(yml, e), f4get(zml, e)};
                            res[e] = resid_cell(L, plain, uni, i + e, j, k, id + e, ch[e], cl[e], hP, lP, hM, lM, bb[e],
                                                bb2[e], bm, bml);
                            acc[0] += res[e] * res[e];
                        }
                    }
                    *(float4 *)(rout + id) = make_float4(res[0], res[1], res[2], res[3]);
                }
                if (RESTRICT) {
                    const float sx0 = res[0] + res[1], sx1 = res[2] + res[3];
                    const int pb = k & 1;
                    // y pairs of the previous plane: the odd warp's sums, written before this barrier
                    if (k > z0 && (w & 1) == 0 && in) {
                        const float2 o = *(const float2 *)&rbuf[pb ^ 1][w >> 1][2 * lane];
                        cs0 += o.x;
                        cs1 += o.y;
                        if ((k - 1) & 1) {
                            const int ci = i >> 1, cj = j >> 1, ck = (k - 1) >> 1;
                            *(float2 *)(C.r + ci + C.g.n[0] * (cj + C.g.n[1] * ck)) = make_float2(cs0, cs1);
                            cs0 = cs1 = 0.f;
                        }
                    }
                    if (w & 1) {
                        *(float2 *)&rbuf[pb][w >> 1][2 * lane] = make_float2(sx0, sx1);
                    } else {
                        cs0 += sx0;
                        cs1 += sx1;
                    }
                }
                hm = hcv; lm = lcv; hcv = hp; lcv = lp; bv = bn; blv = bln;
                stf = stc;
                stc = sti;
                sti = sti + 1 == P ? 0 : sti + 1;
            }
            if (RESTRICT) {
                // the last plane's y pairs (z1 - 1 is odd: the coarse cells complete)
                __syncthreads();
                if ((w & 1) == 0 && in) {
                    const float2 o = *(const float2 *)&rbuf[(z1 - 1) & 1][w >> 1][2 * lane];
                    cs0 += o.x;
                    cs1 += o.y;
                    const int ci = i >> 1, cj = j >> 1, ck = (z1 - 1) >> 1;
                    *(float2 *)(C.r + ci + C.g.n[0] * (cj + C.g.n[1] * ck)) = make_float2(cs0, cs1);
                }
            }
        };
        if (all_uni) march(std::true_type{});
        else march(std::false_type{});
        cpa_wait<0>();
        __syncthreads();
    }
    double out[1];
    if (grid_reduce<1, false, float>(acc, part, &S->counters[RS_RESID], out)) {
        if (threadIdx.x == 0) {
            S->rnorm2 = out[0];
            const double bn = S->bnorm;
            const double rel = bn > 0 ? sqrt(out[0]) / bn : (out[0] > 0 ? 1e300 : 0.0);
            S->rel = rel;
            if (!(rel == rel) || !(bn == bn) || rel >= 1e300) S->status |= 1;
        }
    }
}
