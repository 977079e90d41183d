// wl_common.cuh -- shared device definitions of the BDIM step kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define WL_MAXLEV 16
#define WL_MAXPART 2048  // partial-sum slots per reduction (>= max grid size)

// Grid of one multigrid level (or the fine grid). Periodic axes wrap; on a
// non-periodic axis the normal face of the upper boundary is implicit
// (velocity U_a or the stored exit plane; Poisson coefficient 0).
struct GridD {
    int ndim;
    int n[3];
    int per[3];
    int exit_x;
    long long nc;
    double U[3];
    double nu;
};

__host__ __device__ __forceinline__ long long lin3(const GridD &g, int i, int j, int k) {
    return (long long)i + (long long)g.n[0] * ((long long)j + (long long)g.n[1] * (long long)k);
}

__device__ __forceinline__ void decode(const GridD &g, long long idx, int &i, int &j, int &k) {
    long long q = idx / g.n[0];
    i = (int)(idx - q * g.n[0]);
    k = (int)(q / g.n[1]);
    j = (int)(q - (long long)k * g.n[1]);
}

__device__ __forceinline__ int wrapi(int i, int N) {
    int r = i % N;
    return r < 0 ? r + N : r;
}

// Velocity component a sampled at cell index (i,j,k) with the boundary rule:
// periodic axes wrap; tangential components clamp to the interior (zero
// gradient); the normal component has faces 0..N_a with face N_a the upper
// boundary face (U_a, or the exit plane for u_x when exit_x), clamped there.
template <typename T>
__device__ __forceinline__ T vel_sample(const GridD &g, const T *__restrict__ ua, const T *__restrict__ ue,
                                        int a, int i, int j, int k) {
    int I[3] = {i, j, k};
    bool up = false;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax >= g.ndim) { I[ax] = 0; continue; }
        const int N = g.n[ax];
        if (g.per[ax]) {
            I[ax] = wrapi(I[ax], N);
        } else if (ax == a) {
            if (I[ax] < 0) I[ax] = 0;
            else if (I[ax] >= N) { I[ax] = N; up = true; }
        } else {
            I[ax] = I[ax] < 0 ? 0 : (I[ax] > N - 1 ? N - 1 : I[ax]);
        }
    }
    if (up) return (a == 0 && g.exit_x) ? ue[I[1] + (long long)g.n[1] * I[2]] : (T)g.U[a];
    return ua[lin3(g, I[0], I[1], I[2])];
}

// Stored face array sampled with every axis wrapped / clamped to the stored range.
template <typename T>
__device__ __forceinline__ T face_sample(const GridD &g, const T *__restrict__ f, int i, int j, int k) {
    int I[3] = {i, j, k};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (ax >= g.ndim) { I[ax] = 0; continue; }
        const int N = g.n[ax];
        if (g.per[ax]) I[ax] = wrapi(I[ax], N);
        else I[ax] = I[ax] < 0 ? 0 : (I[ax] > N - 1 ? N - 1 : I[ax]);
    }
    return f[lin3(g, I[0], I[1], I[2])];
}

// Shared-memory address of a generic pointer to shared memory (for PTX).
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum (or max) of K per-thread values of type TA (float partials
// stay float through the warp stage; the cross-warp stage runs in double).
// Result valid in thread 0. `sh` holds >= 32*K doubles.
template <int K, bool MAX, typename TA>
__device__ __forceinline__ void block_reduce(const TA (&v)[K], double (&res)[K], double *sh) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, w = tid >> 5, nw = (nt + 31) >> 5;
    TA x[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        x[q] = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            TA y = __shfl_xor_sync(0xffffffffu, x[q], o);
            x[q] = MAX ? (x[q] > y ? x[q] : y) : x[q] + y;
        }
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < K; ++q) sh[w * K + q] = (double)x[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double y = lane < nw ? sh[lane * K + q] : (MAX ? -1e300 : 0.0);
            res[q] = MAX ? warp_max(y) : warp_sum(y);
        }
    }
    __syncthreads();
}

// Grid-wide deterministic reduction: each block stores its partial, the last
// block to finish combines the partials in block order. Returns true in every
// thread of the last block; then `out` (K values) is valid in thread 0.
// part: K*WL_MAXPART doubles; counter: one unsigned, zero between launches.
template <int K, bool MAX, typename TA>
__device__ __forceinline__ bool grid_reduce(const TA (&v)[K], double *part, unsigned *counter, double (&out)[K]) {
    __shared__ double sh[32 * K];
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    double bv[K];
    block_reduce<K, MAX, TA>(v, bv, sh);
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) part[q * WL_MAXPART + blockIdx.x] = bv[q];
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = MAX ? -1e300 : 0.0;
    for (int b = tid; b < (int)gridDim.x; b += nt)
#pragma unroll
        for (int q = 0; q < K; ++q) {
            double x = ((volatile double *)part)[q * WL_MAXPART + b];
            acc[q] = MAX ? fmax(acc[q], x) : acc[q] + x;
        }
    block_reduce<K, MAX, double>(acc, out, sh);
    if (tid == 0) *counter = 0u;
    return true;
}

// Device-resident scalars of the step and the solver (no host round trip).
struct DevScalars {
    // Poisson right-hand side statistics (mean-free over active rows)
    double bsum, bsq, bmean, bnorm, nact;
    // outer refinement
    double rnorm2, rel;
    int status;              // bit 0: non-finite residual seen
    int pad;
    // PCG scalars per level
    double rho[WL_MAXLEV], alpha[WL_MAXLEV], beta[WL_MAXLEV];
    // step scalars
    double maxflux, dt_next;
    double exit_corr;
    double pmean;
    double red[8];           // general reduction results
    unsigned counters[32];   // one counter per reduction site
};

enum RedSite {
    RS_DIV = 0, RS_RESID, RS_INIT, RS_Q, RS_U, RS_CFL, RS_INVD, RS_PMEAN,
    RS_FORCE, RS_DIAG, RS_MISC
};

template <typename T> struct Vec3P { T *p[3]; };
template <typename T> struct CVec3P { const T *p[3]; };
