// k_flux.cuh -- convection-diffusion flux, Heun stage update and (body-free)
// boundary condition in one shared-memory-tiled kernel.
//
// Sec. 2 (momentum equation F-dot, finite volume on the staggered grid, central
// diffusion, flux-limited QUICK convection, predictor-corrector in time).
// For u_a and direction b the flux through the lower b-face of the u_a control
// volume of cell I is
//     F = Uf * phi - nu (u_a[I] - u_a[I-e_b]),  Uf = (u_b[I] + u_b[I-e_a]) / 2,
// phi the limited QUICK value of u_a upwind of Uf, and
//     r_a[I] = sum_b F_ab(I) - F_ab(I+e_b).
// Every tile stages the velocity with a 2-cell halo in shared memory; tiles
// away from the domain edge copy straight rows, edge tiles apply the boundary
// rule of vel_sample.
#pragma once
#include "wl_common.cuh"

template <int NDIM> struct FluxTile {
    static constexpr int TX = 32;
    static constexpr int TY = NDIM == 3 ? 4 : 8;
    static constexpr int TZ = NDIM == 3 ? 4 : 1;
    static constexpr int H = 2;
    static constexpr int SX = TX + 2 * H;
    static constexpr int SY = TY + 2 * H;
    static constexpr int SZ = NDIM == 3 ? TZ + 2 * H : 1;
    static constexpr int SN = SX * SY * SZ;
    static constexpr int NT = TX * TY * TZ;
};

enum FluxMode {
    FM_RAW = 0,        // out = r (no time step)
    FM_PRED_F = 1,     // out = u0 + dt r                       (u evaluated = u0)
    FM_PRED_U = 2,     // out = BC(u0 + dt r)                   (no body)
    FM_CORR_F = 3,     // out = u0 + dt r(u*)                   (u evaluated = u*)
    FM_CORR_U = 4,     // out = BC((u* + u0 + dt r(u*)) / 2)    (no body)
    // with a body, k_flux4 only: cells of tiles flagged uniform (no body face
    // within a cell of the tile) get the stage's final value, as FM_PRED_U /
    // FM_CORR_U; the others get the blend input, as FM_PRED_F / FM_CORR_F
    FM_PRED_M = 5,
    FM_CORR_M = 6
};

template <typename T> struct FluxArgs {
    const T *u[3];   // velocity at which R is evaluated
    const T *ue;     // its exit plane (may be null when no exit)
    const T *u0[3];  // start-of-step velocity (corrector modes)
    T *out[3];
    T dt;
    const unsigned char *tflag;   // uniform flags of the 32 x 8 x 8 tiles (mixed modes)
    int tntx, tnty;               // tiles along x and y
};

template <typename T>
__device__ __forceinline__ T median3(T a, T b, T c) {
    return max(min(a, b), min(max(a, b), c));
}

// Limited QUICK face value from far-upstream uu, upstream c, downstream d.
template <typename T>
__device__ __forceinline__ T quick_lim(T uu, T c, T d) {
    const T phi = (T(5) * c + T(2) * d - uu) * T(1.0 / 6.0);
    return median3(phi, c, median3(T(10) * c - T(9) * uu, c, d));
}

// Flux of component a (samples sa) along b through the lower b-face of the
// control volume at smem offset L; da/db are smem strides of axes a and b.
template <typename T>
__device__ __forceinline__ T face_flux(const T *__restrict__ sa, const T *__restrict__ sb, int L, int da, int db, T nu) {
    const T Uf = T(0.5) * (sb[L] + sb[L - da]);
    const T sm2 = sa[L - 2 * db], sm1 = sa[L - db], s0 = sa[L], sp1 = sa[L + db];
    const bool pos = Uf > T(0);
    const T uu = pos ? sm2 : sp1;
    const T c = pos ? sm1 : s0;
    const T d = pos ? s0 : sm1;
    return Uf * quick_lim(uu, c, d) - nu * (s0 - sm1);
}

template <typename T, int NDIM, int MODE>
__global__ void __launch_bounds__(FluxTile<NDIM>::NT) k_flux(GridD g, FluxArgs<T> A) {
    using TL = FluxTile<NDIM>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *s = reinterpret_cast<T *>(smraw);
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = tx + TL::TX * (ty + TL::TY * tz);
    const int n0 = g.n[0], n1 = g.n[1], n2 = NDIM == 3 ? g.n[2] : 1;
    const int ntx = (n0 + TL::TX - 1) / TL::TX, nty = (n1 + TL::TY - 1) / TL::TY;
    const int ntz = (n2 + TL::TZ - 1) / TL::TZ;
    const long long ntiles = (long long)ntx * nty * ntz;
    const T nu = (T)g.nu;
    constexpr int st[3] = {1, TL::SX, TL::SX * TL::SY};

    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int bx = (int)(t % ntx);
        const int by = (int)((t / ntx) % nty);
        const int bz = (int)(t / ((long long)ntx * nty));
        const int x0 = bx * TL::TX, y0 = by * TL::TY, z0 = bz * TL::TZ;
        __syncthreads();  // previous tile's readers are done
        // stage the tile row by row (a row: SX samples along x): the threads
        // of one x-row of the block take a staged row each, lanes 0..2H-1 also
        // its last 2H samples. Indices wrap on periodic axes (a shift of at
        // most H); samples beyond a non-periodic domain edge take the
        // boundary rule of vel_sample. Every load of a component is issued
        // before its shared-memory stores.
        constexpr int NROW = TL::SY * TL::SZ;
        constexpr int RPI = TL::TY * TL::TZ;            // rows staged per pass
        constexpr int NPASS = (NROW + RPI - 1) / RPI;
        const int r0 = ty + TL::TY * tz;
        auto wrap = [](int v, int N) { return v < 0 ? v + N : (v >= N ? v - N : v); };
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const T *__restrict__ ua = A.u[a];
            T *sa = s + a * TL::SN;
            T v[NPASS][2];
#pragma unroll
            for (int q = 0; q < NPASS; ++q) {
                const int rr = r0 + q * RPI;
                if (rr < NROW) {
                    const int ly = rr % TL::SY, lz = rr / TL::SY;
                    int gy = y0 + ly - TL::H;
                    int gz = NDIM == 3 ? z0 + lz - TL::H : 0;
                    bool ok = true;
                    if (gy < 0 || gy >= n1) { if (g.per[1]) gy = wrap(gy, n1); else ok = false; }
                    if (NDIM == 3 && (gz < 0 || gz >= n2)) { if (g.per[2]) gz = wrap(gz, n2); else ok = false; }
                    const long long rowb = (long long)n0 * (gy + (long long)n1 * gz);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int lx = h == 0 ? tx : TL::TX + tx;
                        if (h == 1 && tx >= 2 * TL::H) continue;
                        int gx = x0 + lx - TL::H;
                        bool okx = ok;
                        if (gx < 0 || gx >= n0) { if (g.per[0]) gx = wrap(gx, n0); else okx = false; }
                        const int gyr = y0 + ly - TL::H, gzr = NDIM == 3 ? z0 + lz - TL::H : 0;
                        v[q][h] = okx ? ua[gx + rowb] : vel_sample<T>(g, ua, A.ue, a, x0 + lx - TL::H, gyr, gzr);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NPASS; ++q) {
                const int rr = r0 + q * RPI;
                if (rr < NROW) {
                    sa[rr * TL::SX + tx] = v[q][0];
                    if (tx < 2 * TL::H) sa[rr * TL::SX + TL::TX + tx] = v[q][1];
                }
            }
        }
        __syncthreads();
        const int i = x0 + tx, j = y0 + ty, k = z0 + tz;
        if (i >= n0 || j >= n1 || k >= n2) continue;
        const int L = (tx + TL::H) + TL::SX * ((ty + TL::H) + TL::SY * (NDIM == 3 ? tz + TL::H : 0));
        const int idx = i + n0 * (j + n1 * k);
        const int I[3] = {i, j, k};
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            const T *sa = s + a * TL::SN;
            const bool bface = !g.per[a] && I[a] == 0;
            T r = T(0);
#pragma unroll
            for (int b = 0; b < NDIM; ++b) {
                const T *sb = s + b * TL::SN;
                r += face_flux<T>(sa, sb, L, st[a], st[b], nu) - face_flux<T>(sa, sb, L + st[b], st[a], st[b], nu);
            }
            if (bface) r = T(0);
            T outv;
            if (MODE == FM_RAW) {
                outv = r;
            } else if (MODE == FM_PRED_F || MODE == FM_PRED_U) {
                outv = sa[L] + A.dt * r;
                if (MODE == FM_PRED_U && bface) outv = (T)g.U[a];
            } else {
                const T f = A.u0[a][idx] + A.dt * r;
                if (MODE == FM_CORR_F) outv = f;
                else outv = bface ? (T)g.U[a] : T(0.5) * (sa[L] + f);
            }
            A.out[a][idx] = outv;
        }
    }
}
