// wl_static.cu -- small Poisson solve that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a solve:
// an application whose device memory is entirely reserved by its own pool or
// budget, so that a library allocation would fail, or a time-critical loop
// that must not call cudaMalloc because it can synchronise the whole device.
// wl_coarse_solve_static serves them: it solves the same variable-coefficient
// Poisson problem as the library's coarsest multigrid level, with all of its
// working memory in one file-scope device array that every GPU loading the
// library holds until the process exits. The caller passes the coefficients,
// the right-hand side and the output buffer.
#include "../../include/wl.h"
#include "wl_common.cuh"
#include "k_poisson.cuh"

#include <mutex>

// Scratch of the no-allocation solve: 1/D, x, s, d, q (doubles, WL_STATIC_MAX_CELLS
// each) plus 8 result slots. Shared by every call on a device.
static __device__ __align__(256) double wl_static_scratch[5 * WL_STATIC_MAX_CELLS + 8];

namespace {

// The problem of one call: the caller's coefficients, right-hand side and
// output, and the 1/D of every row computed by the kernel into the scratch.
template <typename T>
struct StaticOp {
    GridD g;
    CVec3P<T> c;
    const T *r;
    T *x;
    const double *iD;
    __device__ long long n() const { return g.nc; }
    __device__ double invd(long long e) const { return iD[e]; }
    __device__ double rhs(long long e) const { return (double)r[e]; }
    __device__ double apply(const double *d, long long e) const { return level_apply<T>(g, c.p, d, e); }
    __device__ void out(long long e, double v) const { x[e] = (T)v; }
};

// One block: 1/D in double from the coefficients (upper faces of non-periodic
// axes are 0, periodic axes wrap), then the Jacobi-preconditioned CG of the
// library's coarsest level (block_pcg_solve) on A x = r - mean(r) to rtol or
// maxit; the final relative residual goes to w[5n].
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_static(GridD g, CVec3P<T> cc, const T *r, T *x, double *w, int maxit,
                                                        double rtol) {
    const long long n = g.nc;
    const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    double *iD = w;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const long long q = e / g.n[0];
        const int I[3] = {(int)(e - q * g.n[0]), (int)(q % g.n[1]), (int)(q / g.n[1])};
        double D = 0.0;
        for (int a = 0; a < g.ndim; ++a) {
            const int N = g.n[a];
            const double cp = I[a] + 1 < N ? (double)cc.p[a][e + st[a]]
                                           : (g.per[a] ? (double)cc.p[a][e - (long long)(N - 1) * st[a]] : 0.0);
            D -= cp + (double)cc.p[a][e];
        }
        iD[e] = D != 0.0 ? 1.0 / D : 0.0;
    }
    __syncthreads();
    const double rel = block_pcg_solve(StaticOp<T>{g, cc, r, x, iD}, w + n, w + 2 * n, w + 3 * n, w + 4 * n, maxit, rtol);
    if (threadIdx.x == 0) w[5 * n] = rel;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
double *g_scratch[128] = {};

int scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return WL_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, wl_static_scratch);
        if (e != cudaSuccess || !p) return WL_ERR_CUDA;
        g_scratch[dev] = (double *)p;
    }
    *out = g_scratch[dev];
    return WL_OK;
}

}  // namespace

extern "C" int wl_coarse_solve_static(int ndim, const int *n, const int *periodic, int precision,
                                      const void *const *c, const void *r, void *x, int maxit, double rtol,
                                      void *stream, double *rel_resid) {
    if ((ndim != 2 && ndim != 3) || !n || !c || !r || !x || maxit < 0 || !(rtol >= 0)) return WL_ERR_ARG;
    if (precision != WL_F32 && precision != WL_F64) return WL_ERR_ARG;
    GridD g{};
    g.ndim = ndim;
    long long nc = 1;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = a < ndim ? n[a] : 1;
        g.per[a] = (a < ndim && periodic) ? (periodic[a] != 0) : 0;
        if (g.n[a] < 1) return WL_ERR_ARG;
        nc *= g.n[a];
    }
    for (int a = 0; a < ndim; ++a)
        if (!c[a]) return WL_ERR_ARG;
    if (nc > WL_STATIC_MAX_CELLS) return WL_ERR_ARG;  // beyond the fixed scratch
    g.nc = nc;
    double *w = nullptr;
    int rc = scratch_for_current_device(&w);
    if (rc != WL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = nc >= 4096 ? 1024 : 256;
    if (precision == WL_F32) {
        CVec3P<float> cc{};
        for (int a = 0; a < ndim; ++a) cc.p[a] = (const float *)c[a];
        k_coarse_static<float><<<1, threads, 0, st>>>(g, cc, (const float *)r, (float *)x, w, maxit, rtol);
    } else {
        CVec3P<double> cc{};
        for (int a = 0; a < ndim; ++a) cc.p[a] = (const double *)c[a];
        k_coarse_static<double><<<1, threads, 0, st>>>(g, cc, (const double *)r, (double *)x, w, maxit, rtol);
    }
    if (cudaGetLastError() != cudaSuccess) return WL_ERR_CUDA;
    if (rel_resid) {
        if (cudaMemcpyAsync(rel_resid, w + 5 * nc, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return WL_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return WL_ERR_CUDA;
    }
    return WL_OK;
}
