// k_net_tc.cuh -- the learned guess's 3x3x3 convolution on the fifth-generation
// tensor cores (tcgen05, sm_100 family): per tile of 128 voxels the 27 taps are
// 27 MMAs of M = 128 voxels, N = 16 output channels, K = 16 input channels,
// BF16 operands in shared memory and the FP32 accumulator in tensor memory.
//
// No counterpart in the paper (the network is the learned Poisson guess; the
// paper cites data-driven multigrid, Sec. 3, as precedent). Y = conv(X, W) in
// FP32 (zero padding) and optionally A = relu(Y) in BF16; X: [voxel][16] BF16;
// Wt: [27 taps][16 out][16 in] BF16 (the transposed weights give the
// data-gradient convolution of the backward pass).
//
// Operand layout in shared memory (no swizzle, K-major): 8-row x 16-byte core
// matrices; a row's 16 channels (32 B) span two cores along K, 128 B apart;
// the next 8 rows start 256 B further (the descriptor's leading and stride
// byte offsets). One elected thread issues the MMAs; tcgen05.commit signals a
// per-buffer mbarrier when the MMAs that read that buffer are done, so the
// next tap's voxels are gathered into the other buffer meanwhile. Every wait
// is bounded: on a timeout the kernel sets bit 2 of *status, stops issuing,
// frees its tensor memory and returns.
#pragma once
#include <cstdint>
#include "k_net.cuh"

#define TC_ROWS 128
#define TC_WAIT_TRIES (1 << 20)

__device__ __forceinline__ uint32_t tc_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start, leading byte offset (cores
// adjacent along K), stride byte offset (cores adjacent along M or N), the
// descriptor version (bit 46), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | (uint64_t)((lbo >> 4) & 0x3FFF) << 16 |
           (uint64_t)((sbo >> 4) & 0x3FFF) << 32 | (uint64_t)1 << 46;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 16, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = tc_smem(bar);
    for (int i = 0; i < TC_WAIT_TRIES; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

static __global__ void __launch_bounds__(128) k_conv_fwd_tc(NetGrid g, const __nv_bfloat16 *__restrict__ X,
                                                          const __nv_bfloat16 *__restrict__ Wt,
                                                          float *__restrict__ Y, __nv_bfloat16 *__restrict__ A,
                                                          int *status) {
    __shared__ __align__(1024) uint4 sA[2][TC_ROWS * 2];        // two buffers of 128 rows x 32 B
    __shared__ __align__(1024) uint4 sB[NET_TAPS][NET_C * 2];   // 27 taps x 16 rows x 32 B
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint4 *W4 = reinterpret_cast<const uint4 *>(Wt);
    for (int e = tid; e < NET_TAPS * NET_C * 2; e += blockDim.x) {
        const int t = e / (NET_C * 2), r = e % (NET_C * 2), n = r >> 1, kh = r & 1;
        sB[t][((n >> 3) * 2 + kh) * 8 + (n & 7)] = W4[e];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tc_smem(&tbase)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&mbar[1])));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint4 *X4 = reinterpret_cast<const uint4 *>(X);
    uint32_t parity[2] = {0u, 0u};
    bool pend[2] = {false, false};
    int bad = 0;
    const int ntiles = (g.V + TC_ROWS - 1) / TC_ROWS;
    for (int tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
        const int v = tile * TC_ROWS + tid;
        const bool vok = v < g.V;
        const int q = vok ? v : 0;
        const int x = q % g.nx, y = (q / g.nx) % g.ny, z = q / (g.nx * g.ny);
        for (int t = 0; t < NET_TAPS; ++t) {
            const int b = t & 1;
            // buffer b is free once the MMA that last read it (tap t - 2) is done
            int ok = 1;
            if (tid == 0 && pend[b]) ok = tc_wait(&mbar[b], parity[b]);
            if (__syncthreads_or(!ok)) { bad = 1; break; }
            if (pend[b]) { parity[b] ^= 1u; pend[b] = false; }
            const int nb = vok ? tap_nb(g, x, y, z, t) : -1;
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            sA[b][((tid >> 3) * 2 + 0) * 8 + (tid & 7)] = nb >= 0 ? X4[nb * 2] : zero;
            sA[b][((tid >> 3) * 2 + 1) * 8 + (tid & 7)] = nb >= 0 ? X4[nb * 2 + 1] : zero;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t ad = tc_desc(tc_smem(&sA[b][0]), 128, 256);
                const uint64_t bd = tc_desc(tc_smem(&sB[t][0]), 128, 256);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(t > 0 ? 1 : 0));
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc_smem(&mbar[b]))
                             : "memory");
            }
            pend[b] = true;
        }
        if (bad) break;
        // the tile's accumulator is complete when both buffers' last commits land
        int ok = 1;
        for (int b = 0; b < 2; ++b)
            if (pend[b] && tid == 0) ok &= tc_wait(&mbar[b], parity[b]) ? 1 : 0;
        if (__syncthreads_or(!ok)) { bad = 1; break; }
        for (int b = 0; b < 2; ++b)
            if (pend[b]) { parity[b] ^= 1u; pend[b] = false; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (vok) {
            float4 *y4 = reinterpret_cast<float4 *>(Y + (size_t)v * NET_C);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                y4[c] = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                    __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
            if (A) {
                uint32_t *a32 = reinterpret_cast<uint32_t *>(A) + (size_t)v * (NET_C / 2);
#pragma unroll
                for (int c = 0; c < NET_C / 2; ++c)
                    a32[c] = pack_bf16(fmaxf(__uint_as_float(r[2 * c]), 0.f), fmaxf(__uint_as_float(r[2 * c + 1]), 0.f));
            }
        }
        // the next tile's first MMA overwrites the accumulator: issued only
        // after the barrier that follows these loads
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (bad) {
        // a commit did not arrive in time: wait (bounded) for what was issued,
        // report, and release the tensor memory
        if (tid == 0) {
            for (int b = 0; b < 2; ++b)
                if (pend[b]) tc_wait(&mbar[b], parity[b]);
            atomicOr(status, 4);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// Launch over tiles of 128 voxels (grid-stride; at most 8 blocks per SM of a
// 148-SM part). status: device int whose bit 2 reports a timed-out wait.
inline void conv_fwd_tc(cudaStream_t s, const NetGrid &g, const __nv_bfloat16 *X, const __nv_bfloat16 *Wt, float *Y,
                        __nv_bfloat16 *A, int *status) {
    const int tiles = (g.V + TC_ROWS - 1) / TC_ROWS;
    const int grid = tiles < 1 ? 1 : (tiles < 1184 ? tiles : 1184);
    k_conv_fwd_tc<<<grid, 128, 0, s>>>(g, X, Wt, Y, A, status);
}
