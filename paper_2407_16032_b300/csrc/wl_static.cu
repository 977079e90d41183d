// wl_static.cu -- small Poisson solve that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a solve:
// code that runs while a CUDA graph is being captured (cudaMalloc is not a
// capturable call), or an application whose device memory is entirely
// reserved by its own pool or budget so that a library allocation would fail.
// wl_coarse_solve_static serves them: it solves the same variable-coefficient
// Poisson problem as the library's coarsest multigrid level, with all of its
// working memory in one file-scope device array that every GPU loading the
// library holds until the process exits. The caller passes the coefficients,
// the right-hand side and the output buffer.
#include "../../include/wl.h"
#include "wl_common.cuh"

#include <mutex>

// Scratch of the no-allocation solve: 1/D, x, s, d, q (doubles, WL_STATIC_MAX_CELLS
// each) plus 8 result slots. Shared by every call on a device.
static __device__ __align__(256) double wl_static_scratch[5 * WL_STATIC_MAX_CELLS + 8];

namespace {

// Face coefficient c_a of cell I (lower face) or of its upper neighbour (+1):
// upper faces of non-periodic axes are 0; periodic axes wrap.
template <typename T>
__device__ __forceinline__ double coef(const GridD &g, const T *const *c, int a, const int (&I)[3], long long e,
                                       int up, long long &nb) {
    const long long st[3] = {1, (long long)g.n[0], (long long)g.n[0] * g.n[1]};
    const int N = g.n[a];
    if (up) {
        if (I[a] + 1 < N) { nb = e + st[a]; return (double)c[a][nb]; }
        if (g.per[a]) { nb = e - (long long)(N - 1) * st[a]; return (double)c[a][nb]; }
        nb = e;
        return 0.0;
    }
    if (I[a] > 0) nb = e - st[a];
    else if (g.per[a]) nb = e + (long long)(N - 1) * st[a];
    else nb = e;
    return (double)c[a][e];
}

// One block: Jacobi-preconditioned CG in double on A x = r - mean(r) (mean over
// rows with a nonzero diagonal), to rtol relative residual or maxit iterations;
// writes the mean-free x and, in w[5n], the final relative residual.
template <typename T>
__global__ void k_coarse_static(GridD g, CVec3P<T> cc, const T *r, T *x, double *w, int maxit, double rtol) {
    const long long n = g.nc;
    double *iD = w, *xs = w + n, *ss = w + 2 * n, *ds = w + 3 * n, *qs = w + 4 * n, *res = w + 5 * n;
    __shared__ double sh[64];
    __shared__ double bc[2];  // broadcast of reduction results
    const int tid = threadIdx.x, nt = blockDim.x;
    double v1[1], o1[1], v2[2], o2[2];
    double sr = 0.0, na = 0.0;
    for (long long e = tid; e < n; e += nt) {
        const long long q = e / g.n[0];
        const int I[3] = {(int)(e - q * g.n[0]), (int)(q % g.n[1]), (int)(q / g.n[1])};
        double D = 0.0;
        for (int a = 0; a < g.ndim; ++a) {
            long long nb;
            D -= coef<T>(g, cc.p, a, I, e, 1, nb) + coef<T>(g, cc.p, a, I, e, 0, nb);
        }
        iD[e] = D != 0.0 ? 1.0 / D : 0.0;
        if (D != 0.0) { sr += (double)r[e]; na += 1.0; }
    }
    v2[0] = sr;
    v2[1] = na;
    block_reduce<2, false, double>(v2, o2, sh);
    if (tid == 0) { bc[0] = o2[0]; bc[1] = o2[1]; }
    __syncthreads();
    const double rmean = bc[1] > 0 ? bc[0] / bc[1] : 0.0, nact = bc[1];
    __syncthreads();
    double r0 = 0.0, rho = 0.0;
    for (long long e = tid; e < n; e += nt) {
        const double s = iD[e] != 0.0 ? (double)r[e] - rmean : 0.0;
        xs[e] = 0.0;  // the scratch keeps the previous call's contents: restart from zero
        ss[e] = s;
        ds[e] = iD[e] * s;
        rho += s * ds[e];
        r0 += s * s;
    }
    v2[0] = rho;
    v2[1] = r0;
    block_reduce<2, false, double>(v2, o2, sh);
    if (tid == 0) { bc[0] = o2[0]; bc[1] = o2[1]; }
    __syncthreads();
    rho = bc[0];
    const double rnorm0 = sqrt(bc[1]);
    double sn = rnorm0;
    __syncthreads();
    for (int it = 0; it < maxit && rho != 0.0 && sn > rtol * rnorm0; ++it) {
        double dq = 0.0;
        for (long long e = tid; e < n; e += nt) {
            const long long q = e / g.n[0];
            const int I[3] = {(int)(e - q * g.n[0]), (int)(q % g.n[1]), (int)(q / g.n[1])};
            const double d0 = ds[e];
            double Ad = 0.0;
            for (int a = 0; a < g.ndim; ++a) {
                long long ip, im;
                const double cp = coef<T>(g, cc.p, a, I, e, 1, ip);
                const double cm = coef<T>(g, cc.p, a, I, e, 0, im);
                Ad += cp * (ds[ip] - d0) - cm * (d0 - ds[im]);
            }
            qs[e] = Ad;
            dq += d0 * Ad;
        }
        v1[0] = dq;
        block_reduce<1, false, double>(v1, o1, sh);
        if (tid == 0) bc[0] = o1[0];
        __syncthreads();
        dq = bc[0];
        __syncthreads();
        if (dq == 0.0) break;
        const double alpha = rho / dq;
        double rn = 0.0, s2 = 0.0;
        for (long long e = tid; e < n; e += nt) {
            xs[e] += alpha * ds[e];
            const double s = ss[e] - alpha * qs[e];
            ss[e] = s;
            rn += s * iD[e] * s;
            s2 += s * s;
        }
        v2[0] = rn;
        v2[1] = s2;
        block_reduce<2, false, double>(v2, o2, sh);
        if (tid == 0) { bc[0] = o2[0]; bc[1] = o2[1]; }
        __syncthreads();
        const double rho2 = bc[0];
        sn = sqrt(bc[1]);
        __syncthreads();
        const double beta = rho2 / rho;
        rho = rho2;
        for (long long e = tid; e < n; e += nt) ds[e] = iD[e] * ss[e] + beta * ds[e];
        __syncthreads();
    }
    double sx = 0.0;
    for (long long e = tid; e < n; e += nt)
        if (iD[e] != 0.0) sx += xs[e];
    v1[0] = sx;
    block_reduce<1, false, double>(v1, o1, sh);
    if (tid == 0) bc[0] = o1[0];
    __syncthreads();
    const double xm = nact > 0 ? bc[0] / nact : 0.0;
    for (long long e = tid; e < n; e += nt) x[e] = iD[e] != 0.0 ? (T)(xs[e] - xm) : T(0);
    if (tid == 0) res[0] = rnorm0 > 0 ? sn / rnorm0 : 0.0;
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
