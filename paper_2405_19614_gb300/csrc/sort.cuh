// Internal interface of the onesweep radix-sort passes (sort.cu).
#pragma once

#include "common.cuh"

namespace gs {

constexpr int kSortTileKeys = 4096;  // keys ranked per block of a pass
constexpr int kRadix = 256;

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of one look-back region for passes over up to cap keys: one 256-digit
// row of flags per block of kSortTileKeys keys, plus one.
constexpr size_t onesweep_lookback_bytes(int64_t cap)
{
    return align256(sizeof(uint32_t) * (size_t)((cap + kSortTileKeys - 1) / kSortTileKeys + 1) * kRadix);
}

// Output modes of a pass: separate key and value arrays; (key, value) pairs
// interleaved in kout as uint2; or expanded through SortExpand.
constexpr int kSortPlain = 0, kSortPaired = 1, kSortExpand = 2;

// Where the last pass of the pair sort writes: instead of (key, value) it
// expands each entry (tile, depth rank) into the 64-bit key
// (tile << 32) | rec[rank].x and the value rec[rank].y mod n, where rec holds
// the depth-sorted records as (depth bits, record id).
struct SortExpand {
    uint64_t *keys;
    uint32_t *vals;
    const uint2 *rec;
    uint32_t n;
};

// One stable counting pass of (uint32 key, uint32 value) pairs by the digit
// (key >> shift) & 255, onesweep style: each block ranks 4096 keys in shared
// memory, finds its global offsets by a decoupled look-back over the blocks
// before it, and scatters.  *n_dev (capped at cap) is the key count; hist is
// this digit's histogram over all keys; lb must be zero on entry and lb_next
// is cleared for the pass after.  mode selects the output (kSortPlain,
// kSortPaired into kout, or kSortExpand through expand).  Waits are bounded: a
// look-back that spins too long sets GS_ERR_TIMEOUT in status and moves on.
gs_status_t onesweep_pass(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                          const uint32_t *n_dev, int64_t cap, const uint32_t *hist, uint32_t *lb,
                          uint32_t *lb_next, uint32_t *block_counter, int shift, int mode, const SortExpand *expand,
                          uint32_t *status, cudaStream_t s);

// Adds the digits of the warp's valid keys to shared histograms hist[p][256]
// for the digit passes p < n_passes (8 bits each, from bit 0).  Called by all
// 32 lanes together; a run of equal digits in consecutive lanes is added by
// its first lane in one atomic, so keys that arrive in runs (tile ids of one
// rectangle row, depths of similar magnitude) do not serialise on one bin.
__device__ __forceinline__ void count_digits_warp(uint32_t (*hist)[kRadix], uint32_t key, bool valid, int n_passes)
{
    const int lane = threadIdx.x & 31;
    for (int p = 0; p < n_passes; p++) {
        const uint32_t d = valid ? (key >> (8 * p)) & 0xffu : 0x100u;
        const uint32_t prev = __shfl_up_sync(kFullMask, d, 1);
        const bool head = lane == 0 || prev != d;
        const uint32_t heads = __ballot_sync(kFullMask, head);
        if (head && valid) {
            const uint32_t later = heads & ~((2u << lane) - 1u);  // heads after this lane
            const int next = later ? __ffs(later) - 1 : 32;
            atomicAdd(&hist[p][d], (uint32_t)(next - lane));
        }
    }
}

}  // namespace gs
