// async_copy.cuh -- 16-byte asynchronous copies from global to shared memory
// (cp.async, sm_80 and later) with per-thread commit and wait groups: the
// loads of a later iteration stay in flight without holding registers.
#pragma once

#include <cstdint>

namespace stego {

// 16 bytes from global to shared memory without passing through registers
// (completion per thread through commit and wait groups).
__device__ __forceinline__ void cp_async16(uint4 *smem, const uint4 *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Waits until at most N of the calling thread's committed groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

} // namespace stego
