// paper2.cu -- single-image kernels of the paper's own layout (Sections VI
// and VII: one plane, two bits per cover byte, the message divided greedily
// among rows, pair i of B[j] at A[L*i + j]).  The per-unit, per-run and
// per-row routines live in p2_device.cuh and are shared with the batched
// kernels.
//   p2_embed_units<CH,PLANE,STATS,INPLACE>  persistent grid over 16-pixel
//       units; 256-thread CTAs, each warp's units copied to shared memory
//       one iteration ahead (cp.async).  Out of place one pass (2C + N
//       bytes); in place the units with carrying pixels, read and written
//       back whole.
//   p2_embed_rows  the scatter after a copy (and in place) for layouts the
//       unit kernel does not take; CTAs stride over carrying rows.
//   p2_extract_units<CH,PLANE>  runs of 16 message bytes (CH in {1,3,4}).
//   p2_extract_rows  any channel count.
#include "p2_device.cuh"

namespace stego {
namespace {

// The installed launch shapes are tuned for the one-bit kernels; these
// kernels (other register counts) take as many resident CTAs as occupancy
// allows instead of a tuned CTA count.
constexpr int kAnyCtas = 0;

using p2::View;

struct P2Args {
    View v;
    stego_result *res;
    StatSlot *slot;
};

__device__ __forceinline__ void write_res(const P2Args &a, bool stats)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->msg_bytes = a.v.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
        if (!stats) {
            a.res->changed = 0;
            a.res->sse = 0;
        }
    }
}

constexpr int kUnitThreads = 256; // at most 256: the staging area holds 8 warps
constexpr int kUnitsPerThread = 2;
constexpr int kAsyncUnits = 1; // units per thread and iteration of the copy pipeline (0: off)

// Units one thread takes per iteration of p2_embed_units.
int units_per_thread(uint32_t channels)
{
    return channels > 1 && kAsyncUnits > 0 ? kAsyncUnits : kUnitsPerThread;
}

// Out of place every unit of the image; in place the units with carrying
// pixels.  Three or four channels run the two-stage copy pipeline
// (units_embed_async: 79 registers, three CTAs per SM; 8192x8192x3, plane 0:
// 63.7-65.5 us against 67.6 us with the register-staged units_embed, which
// needed 107-112 registers and two CTAs per SM); one channel loads its
// single-vector units directly.
template <int CH, int PLANE, bool STATS, bool INPLACE>
__global__ void __launch_bounds__(kUnitThreads, 2) p2_embed_units(P2Args a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(a, STATS);
    const uint32_t nunits = a.v.W / 16 * (INPLACE ? a.v.R : a.v.H);
    if constexpr (CH > 1 && kAsyncUnits > 0)
        p2::units_embed_async<CH, PLANE, STATS, kAsyncUnits, INPLACE>(
            a.v, blockIdx.x * blockDim.x * kAsyncUnits + threadIdx.x, nunits,
            gridDim.x * blockDim.x * kAsyncUnits, changed, sse);
    else
        p2::units_embed<CH, PLANE, STATS, kUnitsPerThread, INPLACE>(
            a.v, blockIdx.x * blockDim.x * kUnitsPerThread + threadIdx.x, nunits,
            gridDim.x * blockDim.x * kUnitsPerThread, changed, sse);
    if (STATS)
        block_stats(changed, sse, a.res, a.slot);
}

template <bool STATS>
__global__ void __launch_bounds__(512, 2) p2_embed_rows(P2Args a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    unsigned long long changed = 0, sse = 0;
    write_res(a, STATS);
    p2::rows_embed<STATS>(a.v, blockIdx.x, a.v.R, gridDim.x, changed, sse);
    if (STATS)
        block_stats(changed, sse, a.res, a.slot);
}

__device__ __forceinline__ void extract_res(const P2Args &a)
{
    if (a.res && blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->changed = 0;
        a.res->sse = 0;
        a.res->msg_bytes = a.v.N;
        a.res->status = STEGO_OK;
        a.res->reserved = 0;
    }
}

template <int CH, int PLANE>
__global__ void __launch_bounds__(512) p2_extract_units(P2Args a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    extract_res(a);
    const uint64_t nruns = (uint64_t)((a.v.Q + 15) / 16) * a.v.R;
    p2::runs_extract<CH, PLANE>(a.v, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nruns,
                                (uint64_t)gridDim.x * blockDim.x);
}

__global__ void __launch_bounds__(512) p2_extract_rows(P2Args a)
{
    grid_dependency_wait(); // launched dependent: nothing is touched before
    allow_dependents();
    extract_res(a);
    p2::rows_extract(a.v, blockIdx.x, a.v.R, gridDim.x);
}

P2Args make_args(const uint8_t *src, uint8_t *dst, const stego_geom &g, const uint8_t *msg_in,
                 uint8_t *msg_out, uint64_t N, stego_result *res)
{
    P2Args a;
    a.v = p2::make_view(src, dst, g.width, g.height, g.channels, g.plane, msg_in, msg_out, N);
    a.res = res;
    a.slot = nullptr;
    return a;
}

int row_grid(const void *k, const Shape &sh, uint32_t rows)
{
    return persistent_grid(k, sh.threads, 0, kAnyCtas, rows ? rows : 1, 1);
}

template <bool STATS, bool INPLACE>
const void *units_kernel(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)p2_embed_units<1, 0, STATS, INPLACE>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)p2_embed_units<3, 0, STATS, INPLACE>;
        case 1: return (const void *)p2_embed_units<3, 1, STATS, INPLACE>;
        default: return (const void *)p2_embed_units<3, 2, STATS, INPLACE>;
        }
    }
    switch (plane) {
    case 0: return (const void *)p2_embed_units<4, 0, STATS, INPLACE>;
    case 1: return (const void *)p2_embed_units<4, 1, STATS, INPLACE>;
    case 2: return (const void *)p2_embed_units<4, 2, STATS, INPLACE>;
    default: return (const void *)p2_embed_units<4, 3, STATS, INPLACE>;
    }
}

// Units need 1, 3 or 4 channels, rows of whole 16-byte vectors and a
// 16-byte aligned buffer; unit indices are counted in 32 bits (plus a grid
// stride of headroom).
bool units_layout_ok(const uint8_t *buf, const stego_geom &g)
{
    return (((uintptr_t)buf & 15u) == 0) && p2::unit_channels(g.channels) &&
           g.width % 16u == 0 && (uint64_t)g.width / 16u * g.height < (1ull << 31);
}

const void *extract_units_kernel(uint32_t ch, uint32_t plane)
{
    if (ch == 1)
        return (const void *)p2_extract_units<1, 0>;
    if (ch == 3) {
        switch (plane) {
        case 0: return (const void *)p2_extract_units<3, 0>;
        case 1: return (const void *)p2_extract_units<3, 1>;
        default: return (const void *)p2_extract_units<3, 2>;
        }
    }
    switch (plane) {
    case 0: return (const void *)p2_extract_units<4, 0>;
    case 1: return (const void *)p2_extract_units<4, 1>;
    case 2: return (const void *)p2_extract_units<4, 2>;
    default: return (const void *)p2_extract_units<4, 3>;
    }
}

} // namespace

bool p2_fused_ok(const uint8_t *cover, const uint8_t *stego, const stego_geom &g)
{
    return cover != stego && units_layout_ok(cover, g) && units_layout_ok(stego, g);
}

cudaError_t p2_embed_fused(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                           const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                           const Shape &sh, cudaStream_t s, StatSlot *slot)
{
    P2Args a = make_args(cover, stego, g, msg, nullptr, N, res);
    a.slot = stats ? slot : nullptr;
    const void *k = stats ? units_kernel<true, false>(g.channels, g.plane)
                          : units_kernel<false, false>(g.channels, g.plane);
    const uint64_t nunits = (uint64_t)(g.width / 16u) * g.height;
    const int grid = persistent_grid(k, kUnitThreads, 0, kAnyCtas, nunits ? nunits : 1,
                                     (uint64_t)kUnitThreads * units_per_thread(g.channels));
    void *args[] = {&a};
    return launch_dependent(k, dim3(grid), dim3(kUnitThreads), args, 0, s);
}

cudaError_t p2_embed(const uint8_t *cover, uint8_t *stego, const stego_geom &g,
                     const uint8_t *msg, uint64_t N, bool stats, stego_result *res,
                     const Shape &sh, cudaStream_t s, StatSlot *slot)
{
    P2Args a = make_args(cover, stego, g, msg, nullptr, N, res);
    a.slot = stats ? slot : nullptr;
    if (cover == stego && units_layout_ok(stego, g)) {
        // in place over the units with carrying pixels (cut inside the
        // kernel): whole vectors instead of one byte access per plane byte
        const void *k = stats ? units_kernel<true, true>(g.channels, g.plane)
                              : units_kernel<false, true>(g.channels, g.plane);
        const uint64_t nunits = (uint64_t)(g.width / 16u) * a.v.R;
        const int grid = persistent_grid(k, kUnitThreads, 0, kAnyCtas,
                                         nunits ? nunits : 1,
                                         (uint64_t)kUnitThreads * units_per_thread(g.channels));
        void *args[] = {&a};
        return launch_dependent(k, dim3(grid), dim3(kUnitThreads), args, 0, s);
    }
    const void *k = stats ? (const void *)p2_embed_rows<true> : (const void *)p2_embed_rows<false>;
    const int grid = row_grid(k, sh, a.v.R);
    void *args[] = {&a};
    return launch_dependent(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

cudaError_t p2_extract(const uint8_t *st, const stego_geom &g, uint8_t *msg, uint64_t N,
                       stego_result *res, const Shape &sh, cudaStream_t s)
{
    P2Args a = make_args(st, nullptr, g, nullptr, msg, N, res);
    void *args[] = {&a};
    if (p2::unit_channels(g.channels)) {
        const void *k = extract_units_kernel(g.channels, g.plane);
        const uint64_t runs = (uint64_t)((a.v.Q + 15) / 16) * a.v.R;
        const int grid = persistent_grid(k, sh.threads, 0, kAnyCtas, runs ? runs : 1,
                                         (uint64_t)sh.threads);
        return launch_dependent(k, dim3(grid), dim3(sh.threads), args, 0, s);
    }
    const void *k = (const void *)p2_extract_rows;
    const int grid = row_grid(k, sh, a.v.R);
    return launch_dependent(k, dim3(grid), dim3(sh.threads), args, 0, s);
}

} // namespace stego
