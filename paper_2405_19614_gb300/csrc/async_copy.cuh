// Asynchronous global -> shared copies (cp.async) shared by the kernels that
// stage their inputs in shared memory.
#pragma once

#include <cstdint>

namespace gs {

// 4-byte asynchronous copy global -> shared (Ampere-style cp.async); with
// valid false the source size is 0 and a zero is written instead.
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// 16-byte asynchronous copy global -> shared, bypassing L1; both addresses
// 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// 16-byte asynchronous copy global -> shared through L1 (cached there for
// the next reader); both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16_ca(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Waits until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

}  // namespace gs
