// k_net.cuh -- the learned Poisson initial guess: a small 3D convolutional
// network on a coarse multigrid level, with BF16 tensor-core convolutions and
// FP32 accumulation (the forward and data-gradient convolutions on tcgen05,
// k_net_tc.cuh; the weight gradient here, mma.sync m16n8k16), its backward
// pass and Adam.
//
// No counterpart in the paper (the paper cites data-driven multigrid, Sec. 3,
// as the precedent of learned solver components). Network:
//   h1 = relu(conv(x, W1)), h2 = relu(conv(h1, W2)), y = conv(h2, W3)
// 3x3x3 kernels, zero padding, no biases (so the map is positively homogeneous,
// like the inverse Poisson operator it approximates), channels 1 -> 16 -> 16 -> 1
// held as 16 padded channels throughout (the padded weights are kept at zero).
// Activations: [voxel][16] BF16; weights: [3][27][16 in][16 out] FP32 master
// copy, BF16 working copies laid out [tap][out][in] for the MMA B operand.
#pragma once
#include <cuda_bf16.h>
#include "wl_common.cuh"
#include "k_poisson.cuh"

#define NET_C 16
// Largest grid the network kernels take: they index voxel * NET_C + channel in int.
#define WL_NET_MAX_VOXELS ((long long)(2147483647 / NET_C))
#define NET_TAPS 27
#define NET_WL (NET_TAPS * NET_C * NET_C)  // weights per layer

struct NetGrid {
    int nx, ny, nz, V;
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Neighbour voxel of v at tap t (taps z-major, offsets -1..1), or -1 outside.
__device__ __forceinline__ int tap_nb(const NetGrid &g, int x, int y, int z, int t) {
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int X = x + dx, Y = y + dy, Z = z + dz;
    if (X < 0 || X >= g.nx || Y < 0 || Y >= g.ny || Z < 0 || Z >= g.nz) return -1;
    return X + g.nx * (Y + g.ny * Z);
}

// dW[t][i][o] += sum_v X[v + tap t][i] dZ[v][o] (FP32 atomics). One tap per
// blockIdx.y; each warp reduces chunks of 16 voxels with the MMA (M = 16 input
// channels, N = 16 output channels, K = 16 voxels), staging the transposed
// operands through shared memory.
static __global__ void __launch_bounds__(128) k_conv_dw(NetGrid g, const __nv_bfloat16 *__restrict__ X,
                                                 const __nv_bfloat16 *__restrict__ dZ, float *__restrict__ dW) {
    __shared__ __nv_bfloat16 sx[4][16][18], sd[4][16][18];
    const int t = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int nchunk = (g.V + 15) / 16;
    float d[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int ch = blockIdx.x * 4 + warp; ch < nchunk; ch += gridDim.x * 4) {
        // lane l stages voxel ch*16 + (l & 15), channels 8*(l >> 4) .. +7
        const int v = ch * 16 + (lane & 15), c0 = 8 * (lane >> 4);
        int nb = -1;
        if (v < g.V) {
            const int x = v % g.nx, y = (v / g.nx) % g.ny, z = v / (g.nx * g.ny);
            nb = tap_nb(g, x, y, z, t);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            sx[warp][lane & 15][c0 + c] = nb >= 0 ? X[nb * NET_C + c0 + c] : zero;
            sd[warp][lane & 15][c0 + c] = v < g.V ? dZ[v * NET_C + c0 + c] : zero;
        }
        __syncwarp();
        // A[i][k = voxel], B[k = voxel][o]
        uint32_t a[4];
        __nv_bfloat162 p;
        p.x = sx[warp][2 * tig][gid]; p.y = sx[warp][2 * tig + 1][gid]; a[0] = *reinterpret_cast<uint32_t *>(&p);
        p.x = sx[warp][2 * tig][gid + 8]; p.y = sx[warp][2 * tig + 1][gid + 8]; a[1] = *reinterpret_cast<uint32_t *>(&p);
        p.x = sx[warp][2 * tig + 8][gid]; p.y = sx[warp][2 * tig + 9][gid]; a[2] = *reinterpret_cast<uint32_t *>(&p);
        p.x = sx[warp][2 * tig + 8][gid + 8]; p.y = sx[warp][2 * tig + 9][gid + 8]; a[3] = *reinterpret_cast<uint32_t *>(&p);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            uint32_t b[2];
            p.x = sd[warp][2 * tig][nt * 8 + gid]; p.y = sd[warp][2 * tig + 1][nt * 8 + gid]; b[0] = *reinterpret_cast<uint32_t *>(&p);
            p.x = sd[warp][2 * tig + 8][nt * 8 + gid]; p.y = sd[warp][2 * tig + 9][nt * 8 + gid]; b[1] = *reinterpret_cast<uint32_t *>(&p);
            mma_bf16(d[nt], a, b);
        }
        __syncwarp();
    }
    float *w = dW + t * NET_C * NET_C;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int o = nt * 8 + tig * 2;
        atomicAdd(&w[gid * NET_C + o], d[nt][0]);
        atomicAdd(&w[gid * NET_C + o + 1], d[nt][1]);
        atomicAdd(&w[(gid + 8) * NET_C + o], d[nt][2]);
        atomicAdd(&w[(gid + 8) * NET_C + o + 1], d[nt][3]);
    }
}

// dZ = dA * (Z > 0) in BF16 (ReLU backward), dA and Z FP32.
static __global__ void k_relu_bwd(int n, const float *__restrict__ dA, const float *__restrict__ Z, __nv_bfloat16 *dZ) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        dZ[e] = __float2bfloat16(Z[e] > 0.f ? dA[e] : 0.f);
}

// Network input: channel 0 = x (BF16), other channels 0.
static __global__ void k_net_input(int V, const float *__restrict__ x, __nv_bfloat16 *X) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < NET_C; ++c) X[v * NET_C + c] = __float2bfloat16(c == 0 ? x[v] : 0.f);
}

// Loss sum (y - t)^2 / tn2 of one sample (y = channel 0 of Y) and its gradient
// dY[v][0] = 2 (y - t)/tn2 in BF16 (other channels 0); loss accumulated into
// *loss (FP64 atomics, one per block).
static __global__ void k_net_loss(int V, const float *__restrict__ Y, const float *__restrict__ t, const double *tn2,
                           __nv_bfloat16 *dY, double *loss) {
    __shared__ double sh[64];
    const double den = *tn2 > 0 ? *tn2 : 1.0;
    float acc[1] = {0.f};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        const float e = Y[v * NET_C] - t[v];
        acc[0] += e * e;
#pragma unroll
        for (int c = 0; c < NET_C; ++c) dY[v * NET_C + c] = __float2bfloat16(c == 0 ? (float)(2.0 * e / den) : 0.f);
    }
    double out[1];
    block_reduce<1, false, float>(acc, out, sh);
    if (threadIdx.x == 0) atomicAdd(loss, out[0] / den);
}

// Sum of squares of a sample (its loss normaliser), into *out.
static __global__ void k_sumsq(int V, const float *__restrict__ t, double *out) {
    __shared__ double sh[64];
    float acc[1] = {0.f};
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) acc[0] += t[v] * t[v];
    double o[1];
    block_reduce<1, false, float>(acc, o, sh);
    if (threadIdx.x == 0) atomicAdd(out, o[0]);
}

// BF16 working copies of the FP32 weights W[l][t][i][o]:
// fwd[l][t][o][i] (forward) and bwd[l][t][i][o] = W[l][26 - t][i][o] viewed
// as [t][out = i][in = o] (the transposed, flipped kernel of the dX pass).
static __global__ void k_net_weights(const float *__restrict__ W, __nv_bfloat16 *fwd, __nv_bfloat16 *bwd) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * NET_WL; e += gridDim.x * blockDim.x) {
        const int l = e / NET_WL, r = e % NET_WL;
        const int t = r / (NET_C * NET_C), i = (r / NET_C) % NET_C, o = r % NET_C;
        const __nv_bfloat16 w = __float2bfloat16(W[e]);
        fwd[l * NET_WL + (t * NET_C + o) * NET_C + i] = w;
        bwd[l * NET_WL + ((NET_TAPS - 1 - t) * NET_C + i) * NET_C + o] = w;
    }
}

// Adam step on the FP32 weights (gradients averaged over `nb` samples); the
// padded entries (layer 1 inputs > 0, layer 3 outputs > 0) stay zero.
static __global__ void k_adam(float *W, const float *G, float *m, float *v, int step, float lr, float nb) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * NET_WL; e += gridDim.x * blockDim.x) {
        const int l = e / NET_WL, r = e % NET_WL;
        const int i = (r / NET_C) % NET_C, o = r % NET_C;
        if ((l == 0 && i > 0) || (l == 2 && o > 0)) { W[e] = 0.f; continue; }
        const float gr = G[e] / nb;
        m[e] = b1 * m[e] + (1.f - b1) * gr;
        v[e] = b2 * v[e] + (1.f - b2) * gr * gr;
        W[e] -= lr * (m[e] / c1) / (sqrtf(v[e] / c2) + eps);
    }
}

// Training target of one projection on the coarse level: the mean over each
// coarse cell's fine children of the converged-minus-initial pressure (pairs),
// then mean-free over the coarse grid. Fine (i,j,k) -> coarse (i,j,k) >> s.
template <typename T>
__global__ void k_guess_target(GridD gf, int shift, NetGrid gc, const T *ph1, const T *pl1, const T *ph0,
                               const T *pl0, float *tgt) {
    const int f = 1 << shift;
    const int nfz = gf.ndim == 3 ? f : 1;
    const float inv = 1.f / (float)(f * f * nfz);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < gc.V; v += gridDim.x * blockDim.x) {
        const int x = v % gc.nx, y = (v / gc.nx) % gc.ny, z = v / (gc.nx * gc.ny);
        float s = 0.f;
        for (int dz = 0; dz < nfz; ++dz)
            for (int dy = 0; dy < f; ++dy)
                for (int dx = 0; dx < f; ++dx) {
                    const long long q = lin3(gf, x * f + dx, y * f + dy, gf.ndim == 3 ? z * f + dz : 0);
                    s += (float)((ph1[q] - ph0[q]) + (pl1[q] - pl0[q]));
                }
        tgt[v] = s * inv;
    }
}

// Subtract the mean of a coarse field (one block).
static __global__ void k_demean(int V, float *a) {
    __shared__ double sh[64];
    __shared__ float mean;
    float acc[1] = {0.f};
    for (int v = threadIdx.x; v < V; v += blockDim.x) acc[0] += a[v];
    double o[1];
    block_reduce<1, false, float>(acc, o, sh);
    if (threadIdx.x == 0) mean = (float)(o[0] / V);
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += blockDim.x) a[v] -= mean;
}

// Add the network's coarse correction (channel 0 of Y, times `gain`) to the
// fine refinement pressure, interpolated trilinearly between coarse cell
// centres (wrapped on periodic axes, clamped otherwise): a piecewise-constant
// correction would put steps every 2^shift cells, i.e. a large residual.
template <typename T>
__global__ void k_guess_apply(GridD gf, int shift, NetGrid gc, float gain, const float *__restrict__ Y, T *ph,
                              T *pl) {
    const float f = (float)(1 << shift);
    const int nc[3] = {gc.nx, gc.ny, gc.nz};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < gf.nc;
         q += (long long)gridDim.x * blockDim.x) {
        int I[3];
        decode(gf, q, I[0], I[1], I[2]);
        int c0[3], c1[3];
        float w[3];
        for (int a = 0; a < 3; ++a) {
            if (a >= gf.ndim) { c0[a] = c1[a] = 0; w[a] = 0.f; continue; }
            const float sa = ((float)I[a] + 0.5f) / f - 0.5f;
            const float fl = floorf(sa);
            w[a] = sa - fl;
            int lo = (int)fl, hi = lo + 1;
            if (gf.per[a]) {
                lo = (lo % nc[a] + nc[a]) % nc[a];
                hi = hi % nc[a];
            } else {
                lo = lo < 0 ? 0 : (lo > nc[a] - 1 ? nc[a] - 1 : lo);
                hi = hi < 0 ? 0 : (hi > nc[a] - 1 ? nc[a] - 1 : hi);
            }
            c0[a] = lo;
            c1[a] = hi;
        }
        float val = 0.f;
        for (int corner = 0; corner < 8; ++corner) {
            const int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
            if (gf.ndim == 2 && bz) continue;
            const float wt = (bx ? w[0] : 1.f - w[0]) * (by ? w[1] : 1.f - w[1]) * (gf.ndim == 3 ? (bz ? w[2] : 1.f - w[2]) : 1.f);
            const int v = (bx ? c1[0] : c0[0]) + gc.nx * ((by ? c1[1] : c0[1]) + gc.ny * (bz ? c1[2] : c0[2]));
            val += wt * Y[v * NET_C];
        }
        const T b = (T)(gain * val);
        const T a0 = ph[q];
        const T s = a0 + b, bb = s - a0;
        const T err = (a0 - (s - bb)) + (b - bb);
        const T lo = pl[q] + err, hi = s + lo;
        ph[q] = hi;
        pl[q] = lo - (hi - s);
    }
}

// Small helpers of the guess pipeline.
template <typename T>
__global__ void k_to_float(long long n, const T *__restrict__ a, float *b) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}
static __global__ void k_scale_copy(int n, float s, const float *__restrict__ a, float *b) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) b[e] = s * a[e];
}
static __global__ void k_scale_ch0(int V, float s, float *Y) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) Y[v * NET_C] *= s;
}
static __global__ void k_channel0(int V, const float *__restrict__ Y, float *y) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) y[v] = Y[v * NET_C];
}

// ------------------------------------------------- learned temporal guess
// A 1x1x1 convolution over the pressure history of the same projection stage:
//   guess = H1 + w1 (H1 - H2) + w2 (Ho - H1)
// with H1, H2 the stage's last two converged pressures and Ho the other
// stage's latest (w = (0, 1) is the plain warm start). The weights are fitted
// to the solver's own projections by least squares in the residual norm
// (k_tguess_stats gathers the 2x2 normal equations). Pressures are (hi, lo)
// pairs; the differences are small next to the values and taken in T.
template <typename T>
__global__ void k_tguess_apply(long long n, const T *H1h, const T *H1l, const T *H2h, const T *H2l, const T *Hoh,
                               const T *Hol, T w1, T w2, T *ph, T *pl) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T b = H1h[i], bl = H1l[i];
        const T D1 = (b - H2h[i]) + (bl - H2l[i]);
        const T D2 = (Hoh[i] - b) + (Hol[i] - bl);
        const T c = w1 * D1 + w2 * D2;
        T s, e;
        two_sum(b, c, s, e);
        const T lo = bl + e;
        const T hi = s + lo;
        ph[i] = hi;
        pl[i] = lo - (hi - s);
    }
}

// Normal equations of the fit, for one converged projection P: with
// d = P - H1, D1 = H1 - H2, D2 = Ho - H1, accumulates
//   (A D1)^2, (A D1)(A D2), (A D2)^2, (A D1)(A d), (A D2)(A d), (A d)^2
// over active rows into out[0..5] (the initial residual of the guess is
// A (d - w1 D1 - w2 D2), up to the mean removal).
template <typename T, int NDIM>
__global__ void __launch_bounds__(256) k_tguess_stats(LevelD<T> L, const T *Ph, const T *Pl, const T *H1h,
                                                      const T *H1l, const T *H2h, const T *H2l, const T *Hoh,
                                                      const T *Hol, DevScalars *S, double *part, double *out) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    auto diffs = [&](long long id, double &d, double &D1, double &D2) {
        const double b = (double)H1h[id] + (double)H1l[id];
        d = ((double)Ph[id] + (double)Pl[id]) - b;
        D1 = b - ((double)H2h[id] + (double)H2l[id]);
        D2 = ((double)Hoh[id] + (double)Hol[id]) - b;
    };
    for_cells<NDIM>(L.g, L.tl, L.tflag, [&](int i, int j, int k, long long idx, bool uni) {
        if (!uni && L.invD[idx] == T(0)) return;
        long long ip[3], im[3];
        T cp[3], cm[3];
        nb_setup<T, NDIM>(L, uni, i, j, k, idx, ip, im, cp, cm);
        double d0, a0, b0;
        diffs(idx, d0, a0, b0);
        double Ad = 0, A1 = 0, A2 = 0;
#pragma unroll
        for (int a = 0; a < NDIM; ++a) {
            double dp, ap, bp, dm, am, bm;
            diffs(ip[a], dp, ap, bp);
            diffs(im[a], dm, am, bm);
            const double c1 = (double)cp[a], c0 = (double)cm[a];
            Ad += c1 * (dp - d0) - c0 * (d0 - dm);
            A1 += c1 * (ap - a0) - c0 * (a0 - am);
            A2 += c1 * (bp - b0) - c0 * (b0 - bm);
        }
        acc[0] += A1 * A1;
        acc[1] += A1 * A2;
        acc[2] += A2 * A2;
        acc[3] += A1 * Ad;
        acc[4] += A2 * Ad;
        acc[5] += Ad * Ad;
    });
    double red[6];
    if (grid_reduce<6, false, double>(acc, part, &S->counters[RS_MISC], red))
        if (threadIdx.x == 0 && threadIdx.y == 0)
            for (int q = 0; q < 6; ++q) out[q] += red[q];
}
