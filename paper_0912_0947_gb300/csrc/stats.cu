// stats.cu -- changed-byte count and squared error of two byte arrays, the
// integer quantities behind the PSNR that Section VIII reports:
//   changed = #{k : a[k] != b[k]},  sse = sum (a[k] - b[k])^2,
//   MSE = sse / n,  PSNR = 10 log10(255^2 / MSE).
// Both are exact (64-bit integer accumulation); the host turns them into
// PSNR.  A standalone pass reads 2n bytes; the embed kernels fuse the same
// per-word arithmetic (word_stats) into their store loop at no extra traffic.
#include "internal.cuh"

namespace stego {
namespace {

template <int V>
__global__ void __launch_bounds__(512) changed_vec(const uint4 *__restrict__ a,
                                                    const uint4 *__restrict__ b, uint64_t nvec,
                                                    const uint8_t *a8, const uint8_t *b8,
                                                    uint64_t n, unsigned long long *out)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * V;
    for (uint64_t v0 = (uint64_t)blockIdx.x * blockDim.x * V + threadIdx.x; v0 < nvec;
         v0 += stride) {
        uint4 x[V], y[V];
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v < nvec) {
                x[u] = __ldcs(a + v);
                y[u] = __ldcs(b + v);
            }
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const uint64_t v = v0 + (uint64_t)u * blockDim.x;
            if (v < nvec) {
                word_stats(x[u].x, y[u].x, changed, sse);
                word_stats(x[u].y, y[u].y, changed, sse);
                word_stats(x[u].z, y[u].z, changed, sse);
                word_stats(x[u].w, y[u].w, changed, sse);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < (uint32_t)(n & 15u)) {
        const uint64_t k = (nvec << 4) + threadIdx.x;
        const uint32_t p = a8[k], q = b8[k];
        const uint32_t d = p > q ? p - q : q - p;
        changed += d != 0;
        sse += d * d;
    }
    block_add2(changed, sse, out);
}

__global__ void __launch_bounds__(512) changed_bytes_kernel(const uint8_t *a, const uint8_t *b,
                                                             uint64_t n, unsigned long long *out)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = a[k], q = b[k];
        const uint32_t d = p > q ? p - q : q - p;
        changed += d != 0;
        sse += d * d;
    }
    block_add2(changed, sse, out);
}

} // namespace

cudaError_t changed_bytes(const uint8_t *a, const uint8_t *b, uint64_t n,
                          unsigned long long *out2, const Shape &sh, cudaStream_t s)
{
    const int T = sh.threads;
    if ((((uintptr_t)a | (uintptr_t)b) & 15u) == 0) {
        const uint64_t nvec = n >> 4;
        const void *k;
        switch (sh.vec) {
        case 1: k = (const void *)changed_vec<1>; break;
        case 2: k = (const void *)changed_vec<2>; break;
        case 8: k = (const void *)changed_vec<8>; break;
        default: k = (const void *)changed_vec<4>; break;
        }
        const int vec = (sh.vec == 1 || sh.vec == 2 || sh.vec == 8) ? sh.vec : 4;
        const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, nvec > 0 ? nvec : 1,
                                         (uint64_t)T * vec);
        const uint4 *av = reinterpret_cast<const uint4 *>(a);
        const uint4 *bv = reinterpret_cast<const uint4 *>(b);
        void *args[] = {&av, &bv, (void *)&nvec, &a, &b, &n, &out2};
        return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
    }
    const void *k = (const void *)changed_bytes_kernel;
    const int grid = persistent_grid(k, T, 0, sh.ctas_per_sm, n > 0 ? n : 1, (uint64_t)T * 16);
    void *args[] = {&a, &b, &n, &out2};
    return launch_dependent(k, dim3(grid), dim3(T), args, 0, s);
}

} // namespace stego
