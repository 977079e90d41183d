// k_coarse_dense.cuh -- the coarsest multigrid level (Sec. 2, geometric
// multigrid) by its dense FP64 solution operator on levels of more than 256
// cells. k_coarsest_dense (k_poisson.cuh) does the same product on one block
// for the smaller levels.
#pragma once
#include "k_poisson.cuh"

// The same dense solve for coarsest levels of 257 to WL_DENSE_MAX cells, spread
// over many blocks: FP64 runs at about two FMAs per clock per SM on this part,
// so one block would spend ~n^2/2 clocks on the product. Two launches:
// k_coarsest_dense_rows -- every block forms the active mean of r (the same
//   sum in every block) and r - mean in shared memory; each warp then forms
//   rows of w = M (r - mean), lanes striding over the columns, a shuffle sum;
// k_coarsest_dense_fin -- one block removes the active mean of w and stores
//   it as the level's x.
// w: n doubles of scratch.
#define WL_DENSE_MAX 1024
template <typename T>
__global__ void __launch_bounds__(256) k_coarsest_dense_rows(LevelD<T> L, const double *__restrict__ M,
                                                             double *__restrict__ w) {
    const int n = (int)L.g.nc;
    __shared__ double rr[WL_DENSE_MAX];
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
    const int lane = tid & 31, wpb = nt >> 5;
    for (int e = blockIdx.x * wpb + (tid >> 5); e < n; e += gridDim.x * wpb) {
        const double *row = M + (long long)e * n;
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc = fma(row[c], rr[c], acc);
        acc = warp_sum(acc);
        if (lane == 0) w[e] = acc;
    }
}
template <typename T>
__global__ void __launch_bounds__(256) k_coarsest_dense_fin(LevelD<T> L, const double *__restrict__ w) {
    const int n = (int)L.g.nc;
    __shared__ double sh[64];
    const int tid = threadIdx.x, nt = blockDim.x;
    double v2[2] = {0.0, 0.0}, o2[2];
    for (int e = tid; e < n; e += nt)
        if (L.invD[e] != T(0)) { v2[0] += w[e]; v2[1] += 1.0; }
    block_reduce<2, false, double>(v2, o2, sh);
    if (tid == 0) { sh[40] = o2[0]; sh[41] = o2[1]; }
    __syncthreads();
    const double xm = sh[41] > 0 ? sh[40] / sh[41] : 0.0;
    for (int e = tid; e < n; e += nt) L.x[e] = L.invD[e] != T(0) ? (T)(w[e] - xm) : T(0);
}
