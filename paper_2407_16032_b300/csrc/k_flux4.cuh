// k_flux4.cuh -- convection-diffusion flux and Heun stage update of FP32 3D
// grids on a plane march (Sec. 2: finite volume on the staggered grid,
// central diffusion, flux-limited QUICK convection, predictor-corrector).
//
// For u_a and direction b the flux through the lower b-face of the u_a control
// volume of cell I is
//     F = Uf * phi - nu (u_a[I] - u_a[I-e_b]),  Uf = (u_b[I] + u_b[I-e_a]) / 2,
// phi the limited QUICK value of u_a upwind of Uf, and
//     r_a[I] = sum_b F_ab(I) - F_ab(I+e_b)
// (face_flux and quick_lim of k_flux.cuh, the same arithmetic and order).
//
// A block of 256 threads owns a 128 x 8 tile of the (x, y) plane and marches
// it through KZ planes along z; a thread owns 4 consecutive x cells of one row.
// The three components of each plane, with a ring of 2 cells in x and y, stream
// through five shared stages by per-thread cp.async copies (samples beyond a
// non-periodic domain face are written by the boundary rule of vel_sample).
// Per plane a thread evaluates the x faces of its 4 cells and the one above
// them, the lower and upper y faces of its cells, and the upper z faces of its
// cells, whose values are carried to the next plane as its lower z faces: each
// z-face flux once, the x and y faces at most twice. Four planes (k-1 .. k+2)
// are resident while plane k is finished; one block barrier per plane.
#pragma once
#include "k_flux.cuh"
#include "k_march4.cuh"

namespace f4 {
constexpr int TX = 128, TY = 8;
constexpr int HX = 4, HY = 2;                 // shared rows: HY | TY | HY;  columns: HX | TX | HX
constexpr int RW = TX + 2 * HX;               // 136 floats a row
constexpr int RH = TY + 2 * HY;               // 12 rows
constexpr int CW = RH * RW;                   // one component of a plane
constexpr int SW = 3 * CW;                    // one stage (three components)
constexpr int P = 5;                          // stages
constexpr size_t SMEM = (size_t)P * SW * sizeof(float);
}  // namespace f4

template <int MODE, int KZ>
__global__ void __launch_bounds__(256, 2) k_flux4(GridD g, FluxArgs<float> A) {
    using namespace f4;
    extern __shared__ __align__(16) float fsm[];
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2], plane = n0 * n1;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const float nu = (float)g.nu, dt = A.dt;
    const int ntx = (n0 + TX - 1) / TX, nty = (n1 + TY - 1) / TY, ntz = (n2 + KZ - 1) / KZ;
    for (int t = blockIdx.x; t < ntx * nty * ntz; t += gridDim.x) {
        const int bx = t % ntx, rr = t / ntx, by = rr % nty, bz = rr / nty;
        const int x0 = bx * TX, y0 = by * TY, z0 = bz * KZ;
        const int nx = min(TX, n0 - x0), ny = min(TY, n1 - y0), z1 = min(z0 + KZ, n2);
        const int xb = x0 + 4 * lane, y = y0 + w;
        const bool in = 4 * lane < nx && w < ny;
        const int np = z1 - z0 + 4;   // planes z0-2 .. z1+1 (relative m = 0 .. np-1)
        // the tile touches a non-periodic domain face: ring samples take the boundary rule
        const bool edge = (!px && (x0 == 0 || x0 + nx + 2 > n0)) || (!py && (y0 < 2 || y0 + ny + 2 > n1)) ||
                          (!pz && (z0 < 2 || z1 + 2 > n2));
        // copy (or, beyond a non-periodic face, sample) 16 bytes of component a,
        // shared row r (global row y0 - 2 + r), shared column c (global x0 - 4 + c)
        // of plane gz into stage st
        auto put16 = [&](float *st, int a, int r, int c, int gz) {
            float *dst = st + a * CW + r * RW + c;
            int gy = y0 - HY + r, gx = x0 - HX + c;
            const bool yin = gy >= 0 && gy < n1, zin = gz >= 0 && gz < n2, xin = gx >= 0 && gx + 3 < n0;
            if (!edge || ((yin || py) && (zin || pz) && (xin || px))) {
                gy = yin ? gy : wrapi(gy, n1);
                const int gzz = zin ? gz : wrapi(gz, n2);
                gx = xin ? gx : wrapi(gx, n0);   // a 16-byte group wraps whole: n0 % 4 == 0
                cpa16(dst, A.u[a] + gx + n0 * gy + plane * gzz);
                return;
            }
            // beyond a non-periodic face: the boundary rule of vel_sample (tangential
            // components clamp to the last cell, the normal component to its
            // boundary faces, the upper one carrying U_a or the exit plane)
            bool up = false;
            if (!yin) {
                if (py) gy = wrapi(gy, n1);
                else if (a == 1) { if (gy < 0) gy = 0; else up = true; }
                else gy = gy < 0 ? 0 : n1 - 1;
            }
            if (!zin) {
                if (pz) gz = wrapi(gz, n2);
                else if (a == 2) { if (gz < 0) gz = 0; else up = true; }
                else gz = gz < 0 ? 0 : n2 - 1;
            }
            if (up) {   // the upper boundary face of y or z: U_a
                const float U = (float)g.U[a];
                dst[0] = dst[1] = dst[2] = dst[3] = U;
                return;
            }
            if (xin || px) {   // whole rows of a clamped row / plane
                gx = xin ? gx : wrapi(gx, n0);
                cpa16(dst, A.u[a] + gx + n0 * gy + plane * gz);
                return;
            }
            // a group beyond the x faces: all four samples from one place
            const float *src;
            if (gx < 0) {
                src = A.u[a] + n0 * gy + plane * gz;                       // clamp to x = 0
            } else if (a == 0) {
                if (!g.exit_x) {
                    const float U = (float)g.U[0];
                    dst[0] = dst[1] = dst[2] = dst[3] = U;
                    return;
                }
                src = A.ue + gy + n1 * gz;                                 // exit plane
            } else {
                src = A.u[a] + (n0 - 1) + n0 * gy + plane * gz;            // clamp to x = n0 - 1
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) cpa4(dst + e, src);
        };
        auto issue = [&](int m) {
            if (m < np) {
                float *st = fsm + (m % P) * SW;
                const int gz = z0 - 2 + m;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (in) put16(st, a, w + HY, HX + 4 * lane, gz);
                // ring rows 0, 1, ny + 2, ny + 3 of the three components: 384 groups
                for (int q = tid; q < 384; q += 256) {
                    const int a = q >> 7, rq = (q >> 5) & 3, c = q & 31;
                    const int r = rq < 2 ? rq : ny + rq;
                    if (4 * c < nx) put16(st, a, r, HX + 4 * c, gz);
                }
                // ring columns (groups left and right) of all rows: 2 x RH x 3 groups
                if (tid < 2 * RH * 3) {
                    const int a = tid / (2 * RH), rem = tid % (2 * RH), side = rem & 1, r = rem >> 1;
                    if (r < ny + 2 * HY) put16(st, a, r, side == 0 ? 0 : HX + nx, gz);
                }
            }
            cpa_commit();
        };
        // face fluxes; quick_lim and the upwinding of face_flux (k_flux.cuh)
        auto flux = [&](float Uf, float sm2, float sm1, float s0, float sp1) -> float {
            const bool pos = Uf > 0.f;
            const float uu = pos ? sm2 : sp1, c = pos ? sm1 : s0, d = pos ? s0 : sm1;
            return Uf * quick_lim(uu, c, d) - nu * (s0 - sm1);
        };
        auto row4 = [&](const float *st, int a, int r) {   // own 4 cells of shared row r
            return *(const float4 *)(st + a * CW + r * RW + HX + 4 * lane);
        };
        auto cell = [&](const float *st, int a, int r, int dx) {   // cell xb + dx of shared row r
            return st[a * CW + r * RW + HX + 4 * lane + dx];
        };
        const int ry = w + HY;   // shared row of the thread's cells
        // z faces: the lower z face of plane k (carried) and the upper one
        float fzlo[3][4], fzhi[3][4];
        // flux through the lower z face of relative plane m (planes m-2 .. m+1 resident)
        auto zfaces = [&](int m, float (&out)[3][4]) {
            const float *sa2 = fsm + ((m - 2) % P) * SW, *sa1 = fsm + ((m - 1) % P) * SW;
            const float *s0 = fsm + (m % P) * SW, *sp = fsm + ((m + 1) % P) * SW;
            const float4 uz = row4(s0, 2, ry), uzm1 = row4(sa1, 2, ry);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float4 v2 = row4(sa2, a, ry), v1 = row4(sa1, a, ry), v0 = row4(s0, a, ry), v3 = row4(sp, a, ry);
                float4 ub;   // u_z[I - e_a] on the face plane
                if (a == 0) ub = make_float4(cell(s0, 2, ry, -1), uz.x, uz.y, uz.z);
                else if (a == 1) ub = row4(s0, 2, ry - 1);
                else ub = uzm1;
                const float m2[4] = {v2.x, v2.y, v2.z, v2.w}, m1[4] = {v1.x, v1.y, v1.z, v1.w};
                const float c0[4] = {v0.x, v0.y, v0.z, v0.w}, p1[4] = {v3.x, v3.y, v3.z, v3.w};
                const float zb[4] = {uz.x, uz.y, uz.z, uz.w}, zbm[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) out[a][e] = flux(0.5f * (zb[e] + zbm[e]), m2[e], m1[e], c0[e], p1[e]);
            }
        };
#pragma unroll 1
        for (int m = 0; m < P; ++m) issue(m);
        cpa_wait<1>();   // planes z0-2 .. z0+1
        __syncthreads();
        zfaces(2, fzlo);
        for (int k = z0; k < z1; ++k) {
            const int m = k - z0 + 2;   // relative plane of k
            cpa_wait<0>();              // plane k+2 (issued one plane ago)
            __syncthreads();
            issue(m + 3);               // into the stage of plane k-2, now unused
            const float *sm1 = fsm + ((m - 1) % P) * SW, *s0 = fsm + (m % P) * SW;
            zfaces(m + 1, fzhi);
            float rv[3][4];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // x faces 0..4 at xb .. xb+4: samples xb-2 .. xb+5 of row y
                const float4 c4 = row4(s0, a, ry);
                const float X[8] = {cell(s0, a, ry, -2), cell(s0, a, ry, -1), c4.x, c4.y, c4.z, c4.w,
                                    cell(s0, a, ry, 4), cell(s0, a, ry, 5)};
                // u_x[I] + u_x[I - e_a] on the x faces
                const float4 ux = row4(s0, 0, ry);
                const float UX[5] = {ux.x, ux.y, ux.z, ux.w, cell(s0, 0, ry, 4)};
                float UXm[5];
                if (a == 0) {
                    UXm[0] = cell(s0, 0, ry, -1); UXm[1] = ux.x; UXm[2] = ux.y; UXm[3] = ux.z; UXm[4] = ux.w;
                } else {
                    const float *sb = a == 1 ? s0 : sm1;
                    const int rb = a == 1 ? ry - 1 : ry;
                    const float4 v = row4(sb, 0, rb);
                    UXm[0] = v.x; UXm[1] = v.y; UXm[2] = v.z; UXm[3] = v.w; UXm[4] = cell(sb, 0, rb, 4);
                }
                float fx[5];
#pragma unroll
                for (int f = 0; f < 5; ++f) fx[f] = flux(0.5f * (UX[f] + UXm[f]), X[f], X[f + 1], X[f + 2], X[f + 3]);
                // y faces at y (lower) and y+1 (upper): rows y-2 .. y+2 of the thread's cells
                const float4 Y0 = row4(s0, a, ry - 2), Y1 = row4(s0, a, ry - 1), Y3 = row4(s0, a, ry + 1),
                             Y4 = row4(s0, a, ry + 2);
                const float y0v[4] = {Y0.x, Y0.y, Y0.z, Y0.w}, y1v[4] = {Y1.x, Y1.y, Y1.z, Y1.w};
                const float y2v[4] = {c4.x, c4.y, c4.z, c4.w}, y3v[4] = {Y3.x, Y3.y, Y3.z, Y3.w};
                const float y4v[4] = {Y4.x, Y4.y, Y4.z, Y4.w};
                // u_y[I] + u_y[I - e_a] on the lower and upper y faces
                const float4 uy = row4(s0, 1, ry), uyp = row4(s0, 1, ry + 1);
                float4 uym, uypm;   // u_y[I - e_a] for the lower / upper face
                if (a == 0) {
                    uym = make_float4(cell(s0, 1, ry, -1), uy.x, uy.y, uy.z);
                    uypm = make_float4(cell(s0, 1, ry + 1, -1), uyp.x, uyp.y, uyp.z);
                } else if (a == 1) {
                    uym = row4(s0, 1, ry - 1);
                    uypm = uy;
                } else {
                    uym = row4(sm1, 1, ry);
                    uypm = row4(sm1, 1, ry + 1);
                }
                const float UY[4] = {uy.x, uy.y, uy.z, uy.w}, UYm[4] = {uym.x, uym.y, uym.z, uym.w};
                const float UYp[4] = {uyp.x, uyp.y, uyp.z, uyp.w}, UYpm[4] = {uypm.x, uypm.y, uypm.z, uypm.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float flo = flux(0.5f * (UY[e] + UYm[e]), y0v[e], y1v[e], y2v[e], y3v[e]);
                    const float fhi = flux(0.5f * (UYp[e] + UYpm[e]), y1v[e], y2v[e], y3v[e], y4v[e]);
                    float r = 0.f;
                    r += fx[e] - fx[e + 1];
                    r += flo - fhi;
                    r += fzlo[a][e] - fzhi[a][e];
                    rv[a][e] = r;
                }
            }
            if (in) {
                const int id = xb + n0 * y + plane * k;
                const int I[3] = {xb, y, k};
                // mixed modes: the final value in uniform tiles, the blend input elsewhere
                const bool fin = (MODE == FM_PRED_M || MODE == FM_CORR_M) &&
                                 A.tflag[(xb >> 5) + A.tntx * ((y >> 3) + A.tnty * (k >> 3))] != 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float4 c4 = row4(s0, a, ry);
                    const float sv[4] = {c4.x, c4.y, c4.z, c4.w};
                    float4 u0v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE == FM_CORR_F || MODE == FM_CORR_U || MODE == FM_CORR_M) u0v = *(const float4 *)(A.u0[a] + id);
                    const float u0a[4] = {u0v.x, u0v.y, u0v.z, u0v.w};
                    float o[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const bool bface = !g.per[a] && I[a] + (a == 0 ? e : 0) == 0;
                        const float r = bface ? 0.f : rv[a][e];
                        float outv;
                        if (MODE == FM_RAW) {
                            outv = r;
                        } else if (MODE == FM_PRED_F || MODE == FM_PRED_U || MODE == FM_PRED_M) {
                            outv = sv[e] + dt * r;
                            if ((MODE == FM_PRED_U || (MODE == FM_PRED_M && fin)) && bface) outv = (float)g.U[a];
                        } else {
                            const float f = u0a[e] + dt * r;
                            if (MODE == FM_CORR_F || (MODE == FM_CORR_M && !fin)) outv = f;
                            else outv = bface ? (float)g.U[a] : 0.5f * (sv[e] + f);
                        }
                        o[e] = outv;
                    }
                    *(float4 *)(A.out[a] + id) = make_float4(o[0], o[1], o[2], o[3]);
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int e = 0; e < 4; ++e) fzlo[a][e] = fzhi[a][e];
        }
        cpa_wait<0>();
        __syncthreads();   // every read of the stages is done before the next tile's copies
    }
}
