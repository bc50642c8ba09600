// Tensor-memory-accelerator staging of projected records for the compositing
// kernels: the records of a tile's list are rows of a [rows, 12] FP32 tensor
// (48 bytes each) gathered by index, four rows per cp.async.bulk.tensor
// tile::gather4 instruction, into shared memory, completing on an mbarrier.
//
// Alignment rules kept here: the tensor's base address and row pitch are
// multiples of 16 bytes; the box is one row of 12 floats (48 bytes, a multiple
// of 16) and one row high, as gather4 requires; the column coordinate is 0;
// every shared-memory destination is 128-byte aligned.  Rows are taken from
// the tile lists, so they lie in [0, rows).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace gs {

constexpr int kRecFloats = 12;
constexpr int kRecBytes = 4 * kRecFloats;  // 48
constexpr int kGatherRows = 4;             // rows per gather4
constexpr int kGatherSlot = 256;           // bytes between gather4 destinations (128-byte aligned)
constexpr uint32_t kTmaSpinLimit = 1u << 16;  // tries (each may suspend briefly) before a wait gives up

// A record (row r) lands at slot r % 4 of group r / 4 of a chunk buffer.
__host__ __device__ constexpr int rec_offset(int slot)
{
    return (slot / kGatherRows) * kGatherSlot + (slot % kGatherRows) * kRecBytes;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisations visible to the asynchronous proxy.
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Waits until the barrier's phase with the given parity has completed; gives
// up after kTmaSpinLimit tries (returns false).  A gather completes within
// microseconds; the limit is far beyond that and still ends a broken wait in
// well under a second.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t spins = 0; spins < kTmaSpinLimit; spins++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

// Four rows (r0..r3) of the record tensor into shared memory at dst (128-byte
// aligned), completing on bar.
__device__ __forceinline__ void tma_gather4(void *dst, const CUtensorMap *map, int r0, int r1, int r2, int r3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

// A 4-D box of the tensor into shared memory at dst (128-byte aligned),
// completing on bar; c0 is the innermost coordinate.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// its later asynchronous copies into shared memory.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Host: the tensor map of rows x 12 FP32 records at rec (16-byte aligned).
gs_status_t make_record_map(const float *rec, int64_t rows, CUtensorMap *map);

// Host: a 4-D FP32 tensor map, dims[0] innermost (contiguous), strides[k] the
// bytes between consecutive indices of dimension k + 1 (multiples of 16),
// base 16-byte aligned; out-of-range elements of a box read as zero.
gs_status_t make_tensor_map_4d(const float *base, const uint64_t dims[4], const uint64_t strides[3],
                               const uint32_t box[4], CUtensorMap *map);

}  // namespace gs
